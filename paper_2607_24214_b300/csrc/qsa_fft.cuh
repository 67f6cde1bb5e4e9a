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

}  // namespace qsa
