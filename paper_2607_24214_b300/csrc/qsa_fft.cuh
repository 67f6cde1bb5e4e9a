// Block-cooperative mixed-radix (2, 3, 4) FFT in shared memory.
//
// Self-sorting Stockham formulation (as in Govindaraju et al., "High performance discrete
// Fourier transforms on graphics processors", SC'08): for a stage of radix R after stages
// whose radices multiply to Ns, element j of the n/R butterflies reads x[j + r n/R],
// multiplies input r by W_{Ns R}^{(j mod Ns) r}, does an R-point DFT and writes output r to
// (j / Ns) Ns R + (j mod Ns) + r Ns.  No bit reversal is needed.  `count` independent
// sequences of length n lie back to back; all threads of the block share the butterflies.
// sign = -1 forward (unnormalised), +1 inverse (unnormalised).
#pragma once
#include "qsa_common.cuh"

namespace qsa {

// tw[m] = exp(-2 pi i m / n), m in [0, n); the inverse uses the conjugate.
template <typename R>
__device__ __forceinline__ C<R> twiddle(const C<R>* tw, int m, int sign) {
  C<R> w = tw[m];
  if (sign > 0) w.y = -w.y;
  return w;
}

template <typename R>
__device__ __forceinline__ void dft2(C<R>& a, C<R>& b) {
  C<R> t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <typename R>
__device__ __forceinline__ void dft3(C<R>& a, C<R>& b, C<R>& c, int sign) {
  const R h = R(0.86602540378443864676);  // sqrt(3)/2
  C<R> s = cadd(b, c), d = csub(b, c);
  C<R> m = C<R>{a.x - R(0.5) * s.x, a.y - R(0.5) * s.y};
  // i * sign * h * d
  C<R> e = C<R>{-R(sign) * h * d.y, R(sign) * h * d.x};
  a = cadd(a, s);
  b = cadd(m, e);
  c = csub(m, e);
}

template <typename R>
__device__ __forceinline__ void dft4(C<R>& a, C<R>& b, C<R>& c, C<R>& d, int sign) {
  C<R> s02 = cadd(a, c), d02 = csub(a, c), s13 = cadd(b, d), d13 = csub(b, d);
  // i * sign * d13
  C<R> e = C<R>{-R(sign) * d13.y, R(sign) * d13.x};
  a = cadd(s02, s13);
  c = csub(s02, s13);
  b = cadd(d02, e);
  d = csub(d02, e);
}

// Transforms `count` sequences in buffer a (scratch b); returns the buffer holding the
// result.  Must be called by all threads of the block; synchronises between stages.
template <typename R>
__device__ C<R>* block_fft(C<R>* a, C<R>* b, int count, const FftPlan& plan, const C<R>* tw,
                           int sign) {
  const int n = plan.n;
  for (int s = 0; s < plan.nstages; ++s) {
    const int Rd = plan.radix[s];
    const int Ns = plan.ns[s];
    const int nb = n / Rd;             // butterflies per sequence
    const int stride = n / (Ns * Rd);  // twiddle index step
    const int total = count * nb;
    const int nbsh = plan.nbsh[s], nssh = plan.nssh[s];
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      // index arithmetic with shifts where the sizes are powers of two
      const int seq = nbsh >= 0 ? t >> nbsh : t / nb;
      const int j = t - seq * nb;
      const C<R>* src = a + seq * n;
      C<R>* dst = b + seq * n;
      const int jq = nssh >= 0 ? j >> nssh : j / Ns;
      const int k = j - jq * Ns;
      const int o = jq * Ns * Rd + k;
      if (Rd == 4) {
        C<R> v0 = src[j], v1 = src[j + nb], v2 = src[j + 2 * nb], v3 = src[j + 3 * nb];
        if (k) {
          v1 = cmul(v1, twiddle(tw, k * stride, sign));
          v2 = cmul(v2, twiddle(tw, 2 * k * stride, sign));
          v3 = cmul(v3, twiddle(tw, 3 * k * stride, sign));
        }
        dft4(v0, v1, v2, v3, sign);
        dst[o] = v0;
        dst[o + Ns] = v1;
        dst[o + 2 * Ns] = v2;
        dst[o + 3 * Ns] = v3;
      } else if (Rd == 2) {
        C<R> v0 = src[j], v1 = src[j + nb];
        if (k) v1 = cmul(v1, twiddle(tw, k * stride, sign));
        dft2(v0, v1);
        dst[o] = v0;
        dst[o + Ns] = v1;
      } else {  // 3
        C<R> v0 = src[j], v1 = src[j + nb], v2 = src[j + 2 * nb];
        if (k) {
          v1 = cmul(v1, twiddle(tw, k * stride, sign));
          v2 = cmul(v2, twiddle(tw, 2 * k * stride, sign));
        }
        dft3(v0, v1, v2, sign);
        dst[o] = v0;
        dst[o + Ns] = v1;
        dst[o + 2 * Ns] = v2;
      }
    }
    __syncthreads();
    C<R>* t = a;
    a = b;
    b = t;
  }
  return a;
}

// ------------------------------------------------------------------ one 256-point FFT per warp
// For grids 256 points wide the transforms along x run one per warp, with no block barrier:
// lane l holds x[l + 32 m] (m = 0..7) in registers on entry and X[l + 32 d] (d = 0..7) on
// exit.  With w(N, e) = exp(sign 2 pi i e / N), 256 = 8 x 32 and 32 = 4 x 8 (Cooley-Tukey;
// l = a + 8 b, k2 = c + 4 d):
//   A:  T[l][k1] = w(256, l k1) sum_m x[l + 32 m] w(8, m k1)              in each lane
//   B1: U[k1][a][c] = w(32, a c) sum_b T[a + 8 b][k1] w(4, b c)            lane: (k1, a), two each
//   B2: X[k1 + 8 c + 32 d] = sum_a U[k1][a][c] w(8, a d)                   lane: k1 + 8 c
// and X[k1 + 8 k2] = sum_l T[l][k1] w(32, l k2).  The two regroupings go through the warp's
// buffer F of kWarpFftBuf values: T at F[40 k1 + l], U at F[9 k1 + 72 c + a]; either way a
// half-warp touches 16 distinct bank pairs (one pair of U's store twice).
constexpr int kWarpFftBuf = 320;

// 8-point DFT in registers (natural order in and out): even/odd split into two 4-point DFTs.
template <typename R>
__device__ __forceinline__ void dft8(C<R> (&z)[8], int sign) {
  C<R> e0 = z[0], e1 = z[2], e2 = z[4], e3 = z[6];
  C<R> o0 = z[1], o1 = z[3], o2 = z[5], o3 = z[7];
  dft4(e0, e1, e2, e3, sign);
  dft4(o0, o1, o2, o3, sign);
  const R h = R(0.70710678118654752440);  // 1/sqrt(2)
  const R s = R(sign);
  // O[k] w(8, k): w(8, 1) = (1 + s i)/sqrt 2, w(8, 2) = s i, w(8, 3) = (-1 + s i)/sqrt 2
  const C<R> t1{h * (o1.x - s * o1.y), h * (o1.y + s * o1.x)};
  const C<R> t2{-s * o2.y, s * o2.x};
  const C<R> t3{-h * (o3.x + s * o3.y), h * (s * o3.x - o3.y)};
  z[0] = cadd(e0, o0);
  z[4] = csub(e0, o0);
  z[1] = cadd(e1, t1);
  z[5] = csub(e1, t1);
  z[2] = cadd(e2, t2);
  z[6] = csub(e2, t2);
  z[3] = cadd(e3, t3);
  z[7] = csub(e3, t3);
}

// The 256-point transform of the warp's registers z (see above); F: the warp's kWarpFftBuf
// values of shared memory, tw: the 256-point table.  Called by all 32 lanes.
template <typename R>
__device__ __forceinline__ void warp_fft256(C<R> (&z)[8], C<R>* F, const C<R>* tw, int sign) {
  const int lane = threadIdx.x & 31;
  dft8(z, sign);
#pragma unroll
  for (int k1 = 1; k1 < 8; ++k1) z[k1] = cmul(z[k1], twiddle(tw, lane * k1, sign));
  __syncwarp();  // F is free: the warp's previous reads of it are done
#pragma unroll
  for (int k1 = 0; k1 < 8; ++k1) F[40 * k1 + lane] = z[k1];
  __syncwarp();
  C<R> u[2][4];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int k1 = 4 * h + (lane >> 3), a = lane & 7;
#pragma unroll
    for (int b = 0; b < 4; ++b) u[h][b] = F[40 * k1 + a + 8 * b];
    dft4(u[h][0], u[h][1], u[h][2], u[h][3], sign);
#pragma unroll
    for (int c = 1; c < 4; ++c) u[h][c] = cmul(u[h][c], twiddle(tw, 8 * a * c, sign));
  }
  __syncwarp();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int k1 = 4 * h + (lane >> 3), a = lane & 7;
#pragma unroll
    for (int c = 0; c < 4; ++c) F[9 * k1 + 72 * c + a] = u[h][c];
  }
  __syncwarp();
  {
    const int k1 = lane & 7, c = lane >> 3;
#pragma unroll
    for (int a = 0; a < 8; ++a) z[a] = F[9 * k1 + 72 * c + a];
  }
  dft8(z, sign);
  __syncwarp();  // F may be rewritten by the caller
}

}  // namespace qsa
