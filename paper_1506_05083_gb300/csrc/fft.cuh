// Mixed-radix (4, 2, 3, 5) in-place FFT of one length-P sequence by one warp,
// FP64, for the transforms of the apply: boundary data to modes
// (eq. fhatquad with q = P) and coefficients to point strengths (Sec. 4.1).
//
// Decimation in frequency: with P = r_1 r_2 ... r_m, stage s splits every
// block of length L into r = r_s interleaved sub-sequences, applies the
// r-point DFT across them and the twiddle w_L^{j m}; after the last stage
// position pos(n) holds X[n], where
//   pos(n) = (n mod r_1) (P / r_1) + pos'(n div r_1)
// recursively over the remaining radices (the table `perm` stores pos).
// Twiddles come from the table tw[r] = e^{-2 pi i r / P}.
#pragma once
#include <cuda_runtime.h>

namespace axi {
namespace fft {

constexpr int kMaxStages = 8;

__device__ __forceinline__ double2 c_add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 c_sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 c_mul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 c_mul_mi(double2 a) { return make_double2(a.y, -a.x); }  // -i a

// In-place forward DFT X[n] = sum_l a[l] e^{-2 pi i n l / P}; output in digit-reversed order.
__device__ __forceinline__ void warp_fft(double2 *a, int P, const double2 *__restrict__ tw, const int *rad, int nst,
                         int lane) {
  int L = P;
  for (int s = 0; s < nst; ++s) {
    const int r = rad[s];
    const int Lr = L / r;
    const int stride_tw = P / L;                 // w_L^k = tw[k * P / L]
    const int nb = P / r;                        // butterflies in this stage
    for (int b = lane; b < nb; b += 32) {
      const int blk = b / Lr, j = b % Lr;
      double2 *x = a + blk * L + j;
      if (r == 4) {
        const double2 x0 = x[0], x1 = x[Lr], x2 = x[2 * Lr], x3 = x[3 * Lr];
        const double2 t0 = c_add(x0, x2), t1 = c_sub(x0, x2), t2 = c_add(x1, x3);
        const double2 t3 = c_mul_mi(c_sub(x1, x3));
        const double2 y0 = c_add(t0, t2), y2 = c_sub(t0, t2), y1 = c_add(t1, t3), y3 = c_sub(t1, t3);
        x[0] = y0;
        x[Lr] = c_mul(y1, tw[(j * 1 * stride_tw) % P]);
        x[2 * Lr] = c_mul(y2, tw[(j * 2 * stride_tw) % P]);
        x[3 * Lr] = c_mul(y3, tw[(j * 3 * stride_tw) % P]);
      } else if (r == 2) {
        const double2 x0 = x[0], x1 = x[Lr];
        x[0] = c_add(x0, x1);
        x[Lr] = c_mul(c_sub(x0, x1), tw[(j * stride_tw) % P]);
      } else if (r == 3) {
        // w3 = e^{-2 pi i / 3} = -1/2 - i sqrt(3)/2
        const double h = 0.86602540378443864676;
        const double2 x0 = x[0], x1 = x[Lr], x2 = x[2 * Lr];
        const double2 s12 = c_add(x1, x2), d12 = c_sub(x1, x2);
        const double2 y0 = c_add(x0, s12);
        const double2 m = make_double2(x0.x - 0.5 * s12.x, x0.y - 0.5 * s12.y);
        const double2 rot = make_double2(h * d12.y, -h * d12.x);     // -i sqrt(3)/2 (x1 - x2)
        x[0] = y0;
        x[Lr] = c_mul(c_add(m, rot), tw[(j * stride_tw) % P]);
        x[2 * Lr] = c_mul(c_sub(m, rot), tw[(j * 2 * stride_tw) % P]);
      } else {  // r == 5
        const double c1 = 0.30901699437494742410, c2 = -0.80901699437494742410;  // cos 2pi/5, cos 4pi/5
        const double s1 = 0.95105651629515357212, s2 = 0.58778525229247312917;   // sin 2pi/5, sin 4pi/5
        const double2 x0 = x[0], x1 = x[Lr], x2 = x[2 * Lr], x3 = x[3 * Lr], x4 = x[4 * Lr];
        const double2 a1 = c_add(x1, x4), b1 = c_sub(x1, x4);
        const double2 a2 = c_add(x2, x3), b2 = c_sub(x2, x3);
        const double2 y0 = c_add(x0, c_add(a1, a2));
        const double2 m1 = make_double2(x0.x + c1 * a1.x + c2 * a2.x, x0.y + c1 * a1.y + c2 * a2.y);
        const double2 m2 = make_double2(x0.x + c2 * a1.x + c1 * a2.x, x0.y + c2 * a1.y + c1 * a2.y);
        // -i (s1 b1 + s2 b2) and -i (s2 b1 - s1 b2)
        const double2 n1 = make_double2(s1 * b1.y + s2 * b2.y, -(s1 * b1.x + s2 * b2.x));
        const double2 n2 = make_double2(s2 * b1.y - s1 * b2.y, -(s2 * b1.x - s1 * b2.x));
        x[0] = y0;
        x[Lr] = c_mul(c_add(m1, n1), tw[(j * 1 * stride_tw) % P]);
        x[2 * Lr] = c_mul(c_add(m2, n2), tw[(j * 2 * stride_tw) % P]);
        x[3 * Lr] = c_mul(c_sub(m2, n2), tw[(j * 3 * stride_tw) % P]);
        x[4 * Lr] = c_mul(c_sub(m1, n1), tw[(j * 4 * stride_tw) % P]);
      }
    }
    __syncwarp();
    L = Lr;
  }
}

}  // namespace fft
}  // namespace axi
