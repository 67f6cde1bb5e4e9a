// Shared device helpers of the QS-PIC kernels: complex type, device parameters, bounded grid
// barrier, block reductions, float/double atomics and the Philox-4x32-10 generator.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>
#include <cuda_runtime.h>
#include <stdint.h>

namespace qsa {

template <typename R>
struct C {
  R x, y;
};
template <typename R>
__device__ __forceinline__ C<R> cmk(R a, R b) { return C<R>{a, b}; }
template <typename R>
__device__ __forceinline__ C<R> cadd(C<R> a, C<R> b) { return C<R>{a.x + b.x, a.y + b.y}; }
template <typename R>
__device__ __forceinline__ C<R> csub(C<R> a, C<R> b) { return C<R>{a.x - b.x, a.y - b.y}; }
template <typename R>
__device__ __forceinline__ C<R> cmul(C<R> a, C<R> b) {
  return C<R>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename R>
__device__ __forceinline__ C<R> cconj(C<R> a) { return C<R>{a.x, -a.y}; }
template <typename R>
__device__ __forceinline__ C<R> cscale(C<R> a, R s) { return C<R>{a.x * s, a.y * s}; }
// i * a
template <typename R>
__device__ __forceinline__ C<R> cmuli(C<R> a) { return C<R>{-a.y, a.x}; }

// Status bits latched in the device status word.
enum : int { ST_TIMEOUT = 1, ST_NONFINITE = 2, ST_FLOOR = 4 };

// Largest radix plan: n = 2^a 3^b <= 512 needs at most 9 stages.
constexpr int kMaxStages = 12;

struct FftPlan {
  int n;
  int nstages;
  int radix[kMaxStages];
  int ns[kMaxStages];    // product of the radices of the earlier stages
  int nbsh[kMaxStages];  // log2(n / radix) when a power of two, else -1
  int nssh[kMaxStages];  // log2(ns) when a power of two, else -1
};

// Division of a non-negative int below 2^20 by a fixed divisor d <= 4096 as a multiply-high:
// m = ceil(2^32 / d) makes floor(e m / 2^32) exact there (the error e (m d - 2^32) < 2^32).
struct FastDiv {
  unsigned m;  // 0 for d = 1
};
inline FastDiv make_fastdiv(int d) {
  FastDiv f;
  f.m = d <= 1 ? 0u : (unsigned)((0x100000000ull + (unsigned long long)d - 1) / (unsigned)d);
  return f;
}
__device__ __forceinline__ int div_by(int e, FastDiv f) {
  return f.m ? (int)__umulhi((unsigned)e, f.m) : e;
}
// Division by a small count 1, 2 or 4 (FFT units per block), else a plain division.
__device__ __forceinline__ int div_small(int e, int n) {
  return n == 1 ? e : (n == 2 ? (e >> 1) : (n == 4 ? (e >> 2) : e / n));
}

struct DevParams {
  int nx, ny, nxi, nk;        // nk = nxi + 1 slices/nodes
  int nxh;                    // nx/2 + 1 half-spectrum columns
  int ppx, ppy, ppc, np;      // plasma lattice
  int n_pc;
  double pc_tol2;             // square of the predictor-corrector tolerance (0: fixed n_pc)
  int nsmem_rows;             // tile rows of the plasma deposit (4)
  double Lx, Ly, Lxi, dx, dy, dxi, dt;
  double psi_floor;
  long long spin_limit;
  FftPlan px, py;
  // diagnosed transverse modes: stored at half-spectrum column mkx, row mky; mconj = 1 when
  // the requested k is the conjugate (-k) of the stored one
  int nmodes;
  int mkx[16], mky[16], mconj[16];
  FastDiv fd_nx, fd_ny, fd_nxh;  // division by nx, ny, nx/2 + 1 in the per-element loops
};

// The largest dynamic shared memory a kernel may use is a setting of the function on the
// device, shared by every handle and call in the process: raise it when a launch needs more,
// never lower it (a smaller handle created later must not break a larger one's launches).
inline cudaError_t raise_dyn_smem(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = done[std::make_pair(fn, dev)];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

// ---------------------------------------------------------------------------------------
// Grid-wide barrier for a cooperative launch.  Every wait is bounded by spin_limit polls,
// after which the status word gets ST_TIMEOUT and the barrier reports failure so that every
// block leaves the kernel.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct Barrier {
  unsigned* count;
  int* status;
  long long spin_limit;
};

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned atom_add_acq_rel_u32(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v)
               : "memory");
  return old;
}

// Monotonic arrival counter (zeroed before each launch): the epoch-th barrier of a launch is
// passed once the counter reaches (epoch + 1) * gridDim.x.  Each block's thread 0 adds one
// with acquire-release semantics (publishing the block's writes, ordered by the preceding
// __syncthreads) and polls with acquire loads; the last arriver does not wait.
// Returns true when every block arrived; false (uniformly for the block) on timeout or when
// a timeout was already latched.  arrive (optional): max over blocks of the arrival time.
__device__ __forceinline__ bool grid_sync(const Barrier& b, unsigned& epoch,
                                          unsigned long long* arrive = nullptr) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    if (arrive) atomicMax(arrive, globaltimer());
    int ok = 1;
    const unsigned target = (epoch + 1u) * gridDim.x;
    if (*((volatile int*)b.status) & ST_TIMEOUT) {
      ok = 0;
    } else if (atom_add_acq_rel_u32(b.count, 1u) + 1u != target) {
      long long it = 0;
      while (ld_acquire_u32(b.count) < target) {
        if (++it > b.spin_limit) {
          atomicOr(b.status, ST_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  ++epoch;
  return s_ok != 0;
}

// ---------------------------------------------------------------------------------------
// Block reductions (blockDim.x a multiple of 32, <= 1024).
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_min(T v) {
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// Sum over the block; the result is valid in thread 0.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* scratch /* >= 32 */) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) scratch[w] = v;
  __syncthreads();
  T r = 0;
  if (w == 0) {
    r = (lane < (int)(blockDim.x >> 5)) ? scratch[lane] : T(0);
    r = warp_sum(r);
  }
  return r;
}
// Block reductions whose warp stage runs in the argument's own precision and whose block
// stage runs in FP64 on one thread (FP64 throughput is scarce on this GPU): results valid in
// thread 0; scratch holds >= blockDim/32 doubles (>= N * blockDim/32 for block_sum_lo_n).
template <typename T>
__device__ __forceinline__ double block_sum_lo(T v, double* scratch) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) scratch[w] = (double)v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += scratch[k];
  return r;
}
template <typename T>
__device__ __forceinline__ double block_min_lo(T v, double* scratch) {
  v = warp_min(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) scratch[w] = (double)v;
  __syncthreads();
  double r = scratch[0];
  if (threadIdx.x == 0)
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) r = fmin(r, scratch[k]);
  return r;
}
template <typename T>
__device__ __forceinline__ double block_max_lo(T v, double* scratch) {
  v = warp_max(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) scratch[w] = (double)v;
  __syncthreads();
  double r = scratch[0];
  if (threadIdx.x == 0)
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) r = fmax(r, scratch[k]);
  return r;
}
template <int N, typename T>
__device__ __forceinline__ void block_sum_lo_n(const T v[N], double out[N], double* scratch) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T r[N];
#pragma unroll
  for (int k = 0; k < N; ++k) r[k] = warp_sum(v[k]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < N; ++k) scratch[w * N + k] = (double)r[k];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < N; ++k) {
      double s = 0.0;
      for (int b = 0; b < nw; ++b) s += scratch[b * N + k];
      out[k] = s;
    }
}

// N sums over the block in one exchange (FP64 results, valid in thread 0); scratch >= 32.
template <int N, typename T>
__device__ __forceinline__ void block_sum_n(const T v[N], double out[N], double* scratch) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double r[N];
#pragma unroll
  for (int k = 0; k < N; ++k) r[k] = warp_sum((double)v[k]);
#pragma unroll
  for (int k = 0; k < N; ++k) {
    __syncthreads();
    if (lane == 0) scratch[w] = r[k];
    __syncthreads();
    if (w == 0) out[k] = warp_sum(lane < nw ? scratch[lane] : 0.0);
  }
}

template <typename T>
__device__ __forceinline__ T block_max(T v, T* scratch) {
  v = warp_max(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) scratch[w] = v;
  __syncthreads();
  T r = v;
  if (w == 0) {
    r = (lane < (int)(blockDim.x >> 5)) ? scratch[lane] : scratch[0];
    r = warp_max(r);
  }
  return r;
}
template <typename T>
__device__ __forceinline__ T block_min(T v, T* scratch) {
  v = warp_min(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) scratch[w] = v;
  __syncthreads();
  T r = v;
  if (w == 0) {
    r = (lane < (int)(blockDim.x >> 5)) ? scratch[lane] : scratch[0];
    r = warp_min(r);
  }
  return r;
}

// Non-negative doubles order like their bit patterns: max/min through 64-bit integer atomics.
__device__ __forceinline__ void atomic_max_nonneg(double* p, double v) {
  atomicMax((unsigned long long*)p, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ void atomic_min_nonneg(double* p, double v) {
  atomicMin((unsigned long long*)p, (unsigned long long)__double_as_longlong(v));
}

// ---------------------------------------------------------------------------------------
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): multipliers 0xD2511F53, 0xCD9E8D57,
// Weyl key increments 0x9E3779B9, 0xBB67AE85, ten rounds.
// ---------------------------------------------------------------------------------------
struct U4 {
  uint32_t a, b, c, d;
};
__device__ __forceinline__ U4 philox4x32_10(U4 ctr, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * ctr.a, hi0 = __umulhi(0xD2511F53u, ctr.a);
    const uint32_t lo1 = 0xCD9E8D57u * ctr.c, hi1 = __umulhi(0xCD9E8D57u, ctr.c);
    ctr = U4{hi1 ^ ctr.b ^ k0, lo1, hi0 ^ ctr.d ^ k1, lo0};
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return ctr;
}
__device__ __forceinline__ double u01(uint32_t r) { return ((double)r + 0.5) * (1.0 / 4294967296.0); }

// Asks the L2 cache to fetch `bytes` bytes at p (both multiples of 16) ahead of their use; no
// registers and no shared memory are involved, and nothing waits for it.  Issued in pieces
// of at most 32 KB (multiples of 16 bytes, so every piece stays aligned).
__device__ __forceinline__ void l2_prefetch(const void* p, unsigned bytes) {
  const char* c = static_cast<const char*>(p);
  for (unsigned off = 0; off < bytes; off += 32768u) {
    const unsigned n = bytes - off < 32768u ? bytes - off : 32768u;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(c + off), "r"(n) : "memory");
  }
}

// Shared-memory reduction *addr += v by the lanes whose pred holds, as one predicated
// instruction (no branch around it).
__device__ __forceinline__ void red_shared_if(bool pred, float* addr, float v) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(addr);
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q red.shared.add.f32 [%1], %2;\n\t}"
               ::"r"((int)pred), "r"(sa), "f"(v) : "memory");
}
__device__ __forceinline__ void red_shared_if(bool pred, double* addr, double v) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(addr);
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q red.shared.add.f64 [%1], %2;\n\t}"
               ::"r"((int)pred), "r"(sa), "d"(v) : "memory");
}

// Zero n values at p (shared memory, 16-byte aligned) with 16-byte stores where they fit.
// Called by all threads of the block.
template <typename T>
__device__ __forceinline__ void zero_block(T* p, int n) {
  const int n4 = (int)((size_t)n * sizeof(T) / 16);
  float4* q = reinterpret_cast<float4*>(p);
  for (int e = threadIdx.x; e < n4; e += blockDim.x) q[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int e = (int)(n4 * 16 / sizeof(T)) + threadIdx.x; e < n; e += blockDim.x) p[e] = T(0);
}

// Periodic index: i mod n in [0, n), without a division when i is within one period.
// Bounds checks of the debug build (-DQSA_DEBUG_BOUNDS, libqsa_bounds.so): QSA_IN(cond)
// records the source line of the first failed check and the number of failures, and is
// false when the check fails, so the caller can skip the access.  In the release build it is
// the constant true and costs nothing.  Each translation unit has its own counters; those of
// the file that holds the persistent kernels are read by qsa_bounds_check.
#ifdef QSA_DEBUG_BOUNDS
static __device__ unsigned long long g_bounds_first;
static __device__ unsigned long long g_bounds_count;
__device__ __forceinline__ bool qsa_bounds_fail(int line) {
  atomicCAS(&g_bounds_first, 0ull, (unsigned long long)line);
  atomicAdd(&g_bounds_count, 1ull);
  return false;
}
#define QSA_IN(cond) ((cond) ? true : qsa::qsa_bounds_fail(__LINE__))
#else
#define QSA_IN(cond) true
#endif

__device__ __forceinline__ int wrap(int i, int n) {
  if ((unsigned)i < (unsigned)n) return i;
  if (i < 0 && i >= -n) return i + n;
  if (i >= n && i < 2 * n) return i - n;
  const int r = i % n;
  const int w = r < 0 ? r + n : r;
  (void)QSA_IN(w >= 0 && w < n);
  return w;
}

}  // namespace qsa
