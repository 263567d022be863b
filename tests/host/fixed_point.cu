// Host driver for the exact-arithmetic functions of the gradient product (the same
// header the kernels include, compiled for the CPU).  Reads one case per line from
// stdin and prints the results as integers:
//   w <double bits> <float bits>   -> hi lo E lg neg         (w = r y, FP32 y)
//   W <double bits> <double bits>  -> hi lo E lg neg         (w = r y, FP64 y)
//   x <double bits> <float bits> <ex> -> v0 v1               (to_fx of r y at scale ex)
//   c <v0> <v1> <ex>               -> <FP64 bits> <FP32 bits> (fx_to_f32_f64)
//   l <double bits> <float bits>   -> lg_bound
#include <cstdio>

#include "grad_impl.cuh"

using namespace egt::gradimpl;

int main() {
  char op;
  while (std::scanf(" %c", &op) == 1) {
    if (op == 'w' || op == 'W' || op == 'x') {
      unsigned long long rb, yb;
      int ex = 0;
      if (std::scanf("%llu %llu", &rb, &yb) != 2) return 2;
      if (op == 'x' && std::scanf("%d", &ex) != 1) return 2;
      const double r = bits_f64(rb);
      const WBits w = op == 'W' ? wprod(r, bits_f64(yb)) : wprod(r, bits_f32((unsigned)yb));
      if (op == 'x') {
        const Fx f = to_fx(w, ex);
        std::printf("%lld %lld\n", f.v0, f.v1);
      } else {
        std::printf("%llu %llu %d %d %d\n", w.hi, w.lo, w.E, w.lg, w.neg);
      }
    } else if (op == 'l') {
      unsigned long long rb, yb;
      if (std::scanf("%llu %llu", &rb, &yb) != 2) return 2;
      std::printf("%d\n", lg_bound(bits_f64(rb), bits_f32((unsigned)yb)));
    } else if (op == 'c') {
      long long v0, v1;
      int ex;
      if (std::scanf("%lld %lld %d", &v0, &v1, &ex) != 3) return 2;
      float f;
      double d;
      fx_to_f32_f64(Fx{v0, v1}, ex, f, d);
      std::printf("%llu %u\n", f64_bits(d), f32_bits(f));
    } else {
      return 2;
    }
  }
  return 0;
}
