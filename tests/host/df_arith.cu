// Host-side check of the double-float operations of lqcd_common.cuh (the arithmetic of the
// true-residual kernel): reads pairs of doubles from stdin, prints the double-float sum, product
// and a dot product of each pair's split values as hi lo pairs, for comparison with exact
// rational arithmetic.
#include <cstdio>

#include "lqcd_common.cuh"

using lqcd::dfl;

static dfl split_host(double d) {
  const float hi = (float)d;
  return dfl(hi, (float)(d - (double)hi));
}

int main() {
  double a, b, c;
  while (std::scanf("%lf %lf %lf", &a, &b, &c) == 3) {
    const dfl x = split_host(a), y = split_host(b), z = split_host(c);
    const dfl s = x + y, p = x * y, f = lqcd::fmx(x, y, z);
    const float v[12] = {x.hi, x.lo, y.hi, y.lo, z.hi, z.lo, s.hi, s.lo, p.hi, p.lo, f.hi, f.lo};
    for (int i = 0; i < 12; i++) std::printf("%.17g%c", (double)v[i], i == 11 ? '\n' : ' ');  // exact
  }
  return 0;
}
