// Host driver for the fixed-point functions of the gradient product (the same header
// the kernels include, compiled for the CPU).  Reads one case per line from stdin and
// prints the results as integers:
//   l <double bits> <float bits>          -> lg_bound(r, y)
//   g <double bits>                       -> lg64(w)
//   s <maxlg>                             -> scale_of(maxlg)
//   x <double bits> <float bits> <ex>     -> fixed point of r y 2^ex, FP32 y (fx_of, with
//                                            r_hi, r_lo split from r as the library does)
//   X <double bits> <double bits> <ex>    -> fixed point of r y 2^ex, FP64 y (fx_of64)
//   c <v0> <ex>                           -> <FP64 bits> <FP32 bits> of v0 2^-ex (fx_to_f32_f64)
//   C <v0> <ex>                           -> the same by fx_to_f32_f64_conv
#include <cstdio>

#include "grad_impl.cuh"

using namespace egt::gradimpl;

int main() {
  char op;
  while (std::scanf(" %c", &op) == 1) {
    if (op == 'l') {
      unsigned long long rb, yb;
      if (std::scanf("%llu %llu", &rb, &yb) != 2) return 2;
      std::printf("%d\n", lg_bound(bits_f64(rb), bits_f32((unsigned)yb)));
    } else if (op == 'g') {
      unsigned long long wb;
      if (std::scanf("%llu", &wb) != 1) return 2;
      std::printf("%d\n", lg64(bits_f64(wb)));
    } else if (op == 's') {
      int m;
      if (std::scanf("%d", &m) != 1) return 2;
      std::printf("%d\n", scale_of(m));
    } else if (op == 'x' || op == 'X') {
      unsigned long long rb, yb;
      int ex;
      if (std::scanf("%llu %llu %d", &rb, &yb, &ex) != 3) return 2;
      const double r = bits_f64(rb);
      long long v;
      if (op == 'x') {
        const float r_hi = (float)r, r_lo = (float)(r - (double)r_hi);
        v = fx_of(r, r_hi, r_lo, bits_f32((unsigned)yb), pow2f_split(ex), ex);
      } else {
        v = fx_of64(r, bits_f64(yb), ex);
      }
      std::printf("%lld\n", v);
    } else if (op == 'c' || op == 'C') {
      long long v0;
      int ex;
      if (std::scanf("%lld %d", &v0, &ex) != 2) return 2;
      float f;
      double d;
      if (op == 'c') fx_to_f32_f64(Fx{v0}, ex, f, d);
      else fx_to_f32_f64_conv(Fx{v0}, ex, f, d);
      std::printf("%llu %u\n", f64_bits(d), f32_bits(f));
    } else {
      return 2;
    }
  }
  return 0;
}
