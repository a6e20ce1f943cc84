// The coordinate step of arXiv 2310.16238 §2.4 in double-word arithmetic (dw.cuh): the same
// decisions as ccd_step_rule (ccd_common.cuh), taken on the FP32 pipe, where the scalar step of
// the incremental kernel sits on every coordinate's critical path. Host-compilable, so that the
// CPU tests check it against the oracle's FP64 step.
#pragma once
#include "cox.h"
#include "dw.cuh"

namespace coxgb {

DW_FN bool dw_pos(dw x) { return x.h > 0.0f || (x.h == 0.0f && x.l > 0.0f); }
DW_FN bool dw_negv(dw x) { return x.h < 0.0f || (x.h == 0.0f && x.l < 0.0f); }
DW_FN dw dw_abs(dw x) { return dw_negv(x) ? dw_neg(x) : x; }
DW_FN bool dw_finite(dw x) { return x.h - x.h == 0.0f; }

// The step in FP64: exact -b or +-t where the rule ended there.
DW_FN double inc_step_value(dw s, int kind, double b, double t) {
  return kind == 3 ? -b : kind == 1 ? t : kind == 2 ? -t : dw_to(s);
}

// How a step ended: its computed value, clipped to the trust half-width (+t or -t), or stopped at
// zero (-b, an L1 coefficient that would change sign). The caller takes the exact FP64 t or b for
// the last three: a double-word holds 48 of their 53 bits, and an L1 coefficient must land on an
// exact zero.
enum { kStepValue = 0, kStepPlusT = 1, kStepMinusT = 2, kStepToZero = 3 };

// g1, g2: derivatives of -loglik in the coordinate; b its coefficient (b_zero: exactly 0); t the
// trust half-width; lambda the L1 weight; inv_var the L2 prior's 1/sigma^2. Returns the step and,
// in *kind, how it ended.
DW_FN dw inc_step_rule_dw(dw g1, dw g2, dw b, bool b_zero, dw t, int penalty, dw lambda, dw inv_var, int penalized,
                          int *kind) {
  *kind = kStepValue;
  const bool l1 = penalized && penalty == COX_PEN_L1 && dw_pos(lambda);
  if (penalized && penalty == COX_PEN_L2) {
    g1 = dw_add(g1, dw_mul(b, inv_var));
    g2 = dw_add(g2, inv_var);
  }
  // the Newton numerator of the branch taken (one division below, whichever branch)
  dw num = dw_make(0.0f);
  bool take = false;
  if (dw_pos(g2) && dw_finite(g1) && dw_finite(g2)) {
    if (l1) {
      if (b_zero) {
        const dw up = dw_add(g1, lambda), dn = dw_sub(g1, lambda);
        if (dw_negv(up)) {
          num = up;
          take = true;
        } else if (dw_pos(dn)) {
          num = dn;
          take = true;
        }
      } else {
        num = dw_add(g1, dw_negv(b) ? dw_neg(lambda) : lambda);
        take = true;
      }
    } else {
      num = g1;
      take = true;
    }
  }
  dw s = take ? dw_neg(dw_div(num, g2)) : dw_make(0.0f);
  if (dw_pos(dw_sub(dw_abs(s), t))) {
    *kind = dw_negv(s) ? kStepMinusT : kStepPlusT;
    s = dw_negv(s) ? dw_neg(t) : t;
  }
  if (l1 && !b_zero) {
    const dw nb = dw_add(b, s);
    if ((dw_pos(b) && dw_negv(nb)) || (dw_negv(b) && dw_pos(nb))) {
      *kind = kStepToZero;
      s = dw_neg(b);
    }
  }
  return s;
}

}  // namespace coxgb
