// Reads lines "g1 g2 b t penalty lambda l2_var penalized" (hex doubles / ints), applies the
// incremental kernel's double-word step rule and prints the step as a hex double.
#include <cstdio>

#include "step_rule.cuh"

int main() {
  double g1, g2, b, t, lambda, var;
  int penalty, penalized;
  while (std::scanf("%la %la %la %la %d %la %la %d", &g1, &g2, &b, &t, &penalty, &lambda, &var, &penalized) == 8) {
    using namespace coxgb;
    int kind;
    const dw s = inc_step_rule_dw(dw_from(g1), dw_from(g2), dw_from(b), b == 0.0, dw_from(t), penalty, dw_from(lambda),
                                  dw_from(1.0 / var), penalized, &kind);
    std::printf("%a\n", inc_step_value(s, kind, b, t));
  }
  return 0;
}
