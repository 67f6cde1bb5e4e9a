// qsa_field_solve_static: the transverse field solve of qsa_field_solve, for callers that
// cannot allocate device memory.  See include/qsa.h for the contract.
//
// The scratch memory of the solve (spectra, the interleaved field grid, the deposit buffers
// the row phase reads, twiddle and wavenumber tables, barrier counter, status word) lives in
// one file-scope device array, g_qsa_static_scratch, of QSA_STATIC_SCRATCH_BYTES.  Every GPU
// that loads this library holds that array until the process exits.  Host code cannot use the
// array's name as a device address (the name is a host-side stand-in), so the address is
// taken once per device with cudaGetSymbolAddress, with that device current, on the first
// call made on that device.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/qsa.h"
#include "qsa_common.cuh"
#include "qsa_fft.cuh"
#include "qsa_sweep.cuh"
#include "qsa_tables.h"

using namespace qsa;

namespace qsa {
void set_global_error(const std::string& msg);
}

namespace {

constexpr size_t kStaticBytes = (size_t)QSA_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;
constexpr int kThreadsS = 256;

static __device__ __align__(256) unsigned char g_qsa_static_scratch[kStaticBytes];

std::mutex g_mu;
void* g_base[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set-up on first use).
cudaError_t scratch_base(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_base[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_qsa_static_scratch);
    if (e != cudaSuccess) return e;
    g_base[dev] = p;
  }
  *out = g_base[dev];
  return cudaSuccess;
}

bool static_size_ok(int n) {
  if (n < 1 || n > QSA_STATIC_MAX_N) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

// Every CUDA failure returns QSA_ERR_CUDA with the failing call and CUDA's text in
// qsa_last_error(NULL).
int cuda_err(cudaError_t e, const char* what) {
  set_global_error(std::string("qsa_field_solve_static: ") + what + ": " + cudaGetErrorString(e));
  return QSA_ERR_CUDA;
}

// Bump allocator over the scratch array (offsets only; nothing is allocated).
struct Carve {
  unsigned char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t n) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += n * sizeof(T);
    return p;
  }
};

// Copy the four outputs of the B pass or the three of the psi pass out of the interleaved
// field grid into the caller's arrays; a non-finite output sets ST_NONFINITE in the status word.
template <typename R>
__global__ void extract_kernel(const R* fg, int n, int c0, int nc, R* out0, R* out1, R* out2,
                               R* out3, int* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  R* outs[4] = {out0, out1, out2, out3};
  bool bad = false;
  for (int c = 0; c < nc; ++c) {
    const R v = fg[(size_t)i * kFG + c0 + c];
    outs[c][i] = v;
    bad = bad || !isfinite(v);
  }
  if (bad) atomicOr(status, ST_NONFINITE);
}

template <typename R>
int solve_static(int nx, int ny, double Lx, double Ly, double kappa2, const R* S, const R* Jx,
                 const R* Jy, const R* Jz, const R* Dx, const R* Dy, R* out, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_err(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    set_global_error("qsa_field_solve_static: device ordinal beyond " +
                     std::to_string(kMaxDevices - 1));
    return QSA_ERR_ARG;
  }
  if (st != nullptr) {
    // the scratch array and the launches belong to the current device: so must the stream
    int sdev = -1;
    if ((e = cudaStreamGetDevice(st, &sdev)) != cudaSuccess)
      return cuda_err(e, "cudaStreamGetDevice");
    if (sdev != dev) {
      set_global_error("qsa_field_solve_static: the stream belongs to device " +
                       std::to_string(sdev) + ", not to the current device " +
                       std::to_string(dev));
      return QSA_ERR_ARG;
    }
  }
  void* base = nullptr;
  if ((e = scratch_base(dev, &base)) != cudaSuccess) return cuda_err(e, "cudaGetSymbolAddress");
  DevParams dp{};
  dp.nx = nx;
  dp.ny = ny;
  dp.nxi = 1;
  dp.nk = 1;
  dp.nxh = nx / 2 + 1;
  dp.ppx = dp.ppy = dp.ppc = 1;
  dp.np = nx * ny;
  dp.n_pc = 1;
  dp.nsmem_rows = kTileRows;
  dp.Lx = Lx;
  dp.Ly = Ly;
  dp.Lxi = 1.0;
  dp.dx = Lx / nx;
  dp.dy = Ly / ny;
  dp.dxi = 1.0;  // the D inputs enter as J^{+1/2} = D dxi with J^{-1/2} = 0
  dp.dt = 1.0;
  dp.psi_floor = 0.05;
  dp.spin_limit = 1ll << 26;
  dp.px = make_plan(nx);
  dp.py = make_plan(ny);
  dp.fd_nx = make_fastdiv(nx);
  dp.fd_ny = make_fastdiv(ny);
  dp.fd_nxh = make_fastdiv(dp.nxh);
  const size_t g = (size_t)nx * ny, spec = (size_t)dp.nxh * ny;
  const size_t smem = sweep_smem_bytes<R>(nx, ny);
  int per_sm = 0, sms = 0;
  if ((e = raise_dyn_smem((const void*)solve_kernel<R>, smem)) != cudaSuccess)
    return cuda_err(e, "cudaFuncSetAttribute");
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_kernel<R>, kThreadsS,
                                                         smem)) != cudaSuccess)
    return cuda_err(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return cuda_err(e, "cudaDeviceGetAttribute");
  if (per_sm < 1) {
    set_global_error("qsa_field_solve_static: the solve kernel does not fit on an SM");
    return QSA_ERR_ARG;
  }
  int grid = per_sm * sms;
  const int work = ny > dp.nxh ? ny : dp.nxh;
  if (grid > work) grid = work;

  Carve cv{reinterpret_cast<unsigned char*>(base)};
  SweepArgs<R> a{};
  a.p = dp;
  a.k = sweep_consts<R>(dp);
  a.fg = cv.take<R>(g * kFG);
  a.part = cv.take<R>((size_t)ny * kTileRows * nx * kNF);
  a.ovf = cv.take<R>(g * kNF);
  a.cflag = cv.take<int>((size_t)ny);
  a.odirty = cv.take<int>((size_t)ny);
  a.rspec = cv.take<C<R>>(kNF * spec);
  a.cspec = cv.take<C<R>>(4 * spec);
  a.jprev = cv.take<C<R>>(2 * spec);
  a.bold = cv.take<C<R>>(2 * spec);
  C<R>* tw = cv.take<C<R>>((size_t)nx + ny);
  R* ktab = cv.take<R>((size_t)2 * dp.nxh + 2 * ny);
  a.diag = cv.take<double>((size_t)D_COUNT);
  a.dpart = cv.take<double>((size_t)grid * P_COUNT);
  unsigned* count = cv.take<unsigned>(1);
  int* status = cv.take<int>(1);
  if (cv.off > kStaticBytes) {
    set_global_error("qsa_field_solve_static: scratch for this grid exceeds the static array");
    return QSA_ERR_ARG;
  }
  a.twx = tw;
  a.twy = tw + nx;
  a.ktab = ktab;
  a.src = nullptr;
  a.slab = nullptr;
  a.bref = nullptr;
  a.ptimes = nullptr;
  a.bar = Barrier{count, status, dp.spin_limit};

  // tables, built in FP64 on the host (copied, nothing allocated on the device)
  const std::vector<C<R>> twh = twiddle_table<R>(nx, ny);
  const std::vector<R> kt = wavenumber_table<R>(nx, ny, Lx, Ly);
  std::vector<double> dg(D_COUNT, 0.0);
  dg[D_KAPPA] = kappa2 * (double)nx * ny;  // the solve scales by ppc * nx * ny (ppc = 1)

#define QSA_TRY(x)                                      \
  do {                                                  \
    const cudaError_t e_ = (x);                         \
    if (e_ != cudaSuccess) return cuda_err(e_, #x);     \
  } while (0)
  QSA_TRY(cudaMemcpyAsync(tw, twh.data(), twh.size() * sizeof(C<R>), cudaMemcpyHostToDevice, st));
  QSA_TRY(cudaMemcpyAsync(ktab, kt.data(), kt.size() * sizeof(R), cudaMemcpyHostToDevice, st));
  QSA_TRY(cudaMemcpyAsync(a.diag, dg.data(), dg.size() * sizeof(double), cudaMemcpyHostToDevice,
                          st));
  // state the previous call left behind that must start at zero
  QSA_TRY(cudaMemsetAsync(a.part, 0, (size_t)ny * kTileRows * nx * kNF * sizeof(R), st));
  QSA_TRY(cudaMemsetAsync(a.jprev, 0, 2 * spec * sizeof(C<R>), st));
  QSA_TRY(cudaMemsetAsync(a.bold, 0, 2 * spec * sizeof(C<R>), st));
  QSA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
  // the inputs sit in the overflow grid: every overflow row is read, no outer tile row
  QSA_TRY(cudaMemsetAsync(a.cflag, 0, (size_t)ny * sizeof(int), st));
  QSA_TRY(cudaMemsetAsync(a.odirty, 1, (size_t)ny * sizeof(int), st));
  // B pass: the five trial fields J_x, J_y, J_z, J_x^{+1/2}, J_y^{+1/2}, field-major
  const R* ins[5] = {Jx, Jy, Jz, Dx, Dy};
  for (int f = 0; f < 5; ++f)
    QSA_TRY(cudaMemcpyAsync(a.ovf + (size_t)f * g, ins[f], g * sizeof(R),
                            cudaMemcpyDeviceToDevice, st));
  QSA_TRY(cudaMemsetAsync(count, 0, sizeof(unsigned), st));
  int which = 0;
  void* args[] = {&a, &which};
  QSA_TRY(cudaLaunchCooperativeKernel((void*)solve_kernel<R>, dim3(grid), dim3(kThreadsS), args,
                                      smem, st));
  const unsigned eb = (unsigned)((g + 255) / 256);
  extract_kernel<R><<<eb, 256, 0, st>>>(a.fg, (int)g, FG_BX, 4, out + 5 * g, out + 6 * g,
                                        out + 4 * g, out + 3 * g, status);
  QSA_TRY(cudaGetLastError());
  // psi pass: S in field 0 of three
  QSA_TRY(cudaMemsetAsync(a.ovf, 0, 3 * g * sizeof(R), st));
  QSA_TRY(cudaMemcpyAsync(a.ovf, S, g * sizeof(R), cudaMemcpyDeviceToDevice, st));
  QSA_TRY(cudaMemsetAsync(a.odirty, 1, (size_t)ny * sizeof(int), st));
  QSA_TRY(cudaMemsetAsync(a.part, 0, (size_t)ny * kTileRows * nx * kNF * sizeof(R), st));
  QSA_TRY(cudaMemsetAsync(count, 0, sizeof(unsigned), st));
  which = 1;
  QSA_TRY(cudaLaunchCooperativeKernel((void*)solve_kernel<R>, dim3(grid), dim3(kThreadsS), args,
                                      smem, st));
  extract_kernel<R><<<eb, 256, 0, st>>>(a.fg, (int)g, FG_PSI, 3, out, out + g, out + 2 * g,
                                        nullptr, status);
  QSA_TRY(cudaGetLastError());
  int hst = 0;
  QSA_TRY(cudaMemcpyAsync(&hst, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  QSA_TRY(cudaStreamSynchronize(st));
#undef QSA_TRY
  const int rc = status_code(hst);
  if (rc < 0) {
    set_global_error(std::string("qsa_field_solve_static: ") + status_text(rc));
    return rc;
  }
  return QSA_OK;
}

}  // namespace

extern "C" int qsa_field_solve_static(int32_t nx, int32_t ny, double Lx, double Ly,
                                      double kappa2, int32_t precision, const void* S,
                                      const void* Jx, const void* Jy, const void* Jz,
                                      const void* Dx, const void* Dy, void* out, void* stream) {
  if (!static_size_ok(nx) || !static_size_ok(ny)) {
    set_global_error("qsa_field_solve_static: nx, ny must be 1 or 2^a 3^b and at most " +
                     std::to_string(QSA_STATIC_MAX_N));
    return QSA_ERR_ARG;
  }
  if (!(Lx > 0) || !(Ly > 0) || !(kappa2 >= 0) || !S || !Jx || !Jy || !Jz || !Dx || !Dy || !out) {
    set_global_error("qsa_field_solve_static: invalid box, kappa2 or NULL array");
    return QSA_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == QSA_FP64)
    return solve_static<double>(nx, ny, Lx, Ly, kappa2, (const double*)S, (const double*)Jx,
                                (const double*)Jy, (const double*)Jz, (const double*)Dx,
                                (const double*)Dy, (double*)out, st);
  if (precision == QSA_MIXED)
    return solve_static<float>(nx, ny, Lx, Ly, kappa2, (const float*)S, (const float*)Jx,
                               (const float*)Jy, (const float*)Jz, (const float*)Dx,
                               (const float*)Dy, (float*)out, st);
  set_global_error("qsa_field_solve_static: unknown precision");
  return QSA_ERR_ARG;
}

namespace qsa {
// The bounds-checked debug build's counters of this file (each file compiled without
// separate device linking has its own): read by qsa_bounds_check.
int static_bounds_counts(unsigned long long* first, unsigned long long* count) {
  *first = 0;
  *count = 0;
#ifdef QSA_DEBUG_BOUNDS
  if (cudaMemcpyFromSymbol(first, g_bounds_first, sizeof(*first)) != cudaSuccess ||
      cudaMemcpyFromSymbol(count, g_bounds_count, sizeof(*count)) != cudaSuccess)
    return QSA_ERR_CUDA;
#endif
  return QSA_OK;
}
}  // namespace qsa
