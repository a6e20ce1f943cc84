// Reads lines "op xh xl yh yl" (hex floats), applies the library's double-word operation and
// prints "rh rl" (hex floats). The caller checks the results in exact rational arithmetic.
#include <cstdio>
#include <cstring>

#include "dw.cuh"

using coxgb::dw;

int main() {
  char op[16];
  float xh, xl, yh, yl;
  while (std::scanf("%15s %a %a %a %a", op, &xh, &xl, &yh, &yl) == 5) {
    const dw x{xh, xl}, y{yh, yl};
    dw r{0.0f, 0.0f};
    if (!std::strcmp(op, "add")) r = coxgb::dw_add(x, y);
    else if (!std::strcmp(op, "addsame")) r = coxgb::dw_add_same(x, y);
    else if (!std::strcmp(op, "mul")) r = coxgb::dw_mul(x, y);
    else if (!std::strcmp(op, "mulf")) r = coxgb::dw_mul_f(x, yh);
    else if (!std::strcmp(op, "div")) r = coxgb::dw_div(x, y);
    else if (!std::strcmp(op, "twosum")) r = coxgb::two_sum(xh, yh);
    else if (!std::strcmp(op, "twoprod")) r = coxgb::two_prod(xh, yh);
    std::printf("%a %a\n", double(r.h), double(r.l));
  }
  return 0;
}
