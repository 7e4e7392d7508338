// C-ABI entry points that are not a solver family of their own: version and
// error reporting, instrumentation, the Gibbs operator alone (and its
// no-allocation form), plan application, the objective, and the colour
// transfer steps (Sec. 5.1).  The solvers live in uot_solve.cu (uot_solve,
// uot_solve_many, uot_solve_batch), uot_mass.cu (Algorithm 4), uot_wf.cu (WF
// gradient flows) and uot_bary.cu (barycenters); the host machinery they share
// is in uot_host.cuh.
//
// Every kernel on the path is this library's own; no CPU fallback exists.
#include <map>
#include <mutex>
#include <utility>

#include "uot_host.cuh"

namespace uot {

thread_local std::string g_last_error;
std::atomic<long long> g_launches{0};
Prof g_prof;

namespace {

// ---------------------------------------------------------------------------
// Colour transfer (Sec. 5.1): histograms, barycentric projection, bin map
// ---------------------------------------------------------------------------

constexpr int kMaxBinDim = 8;
struct BinGrid {
  int d;
  int shape[kMaxBinDim];
};

// Row-major bin of a point of [0, 1]^d: bin k of axis a covers [k/n_a, (k+1)/n_a);
// the floor is taken on the FP32 product x * n_a, outside points are clamped
// and NaN goes to bin 0.
__device__ __forceinline__ int64_t bin_of(const float* __restrict__ x, const BinGrid& b) {
  int64_t idx = 0;
  for (int a = 0; a < b.d; ++a) {
    const float v = floorf(__fmul_rn(x[a], (float)b.shape[a]));
    const int k = (v != v || v < 0.0f) ? 0 : (v > (float)(b.shape[a] - 1) ? b.shape[a] - 1 : (int)v);
    idx = idx * b.shape[a] + k;
  }
  return idx;
}

__global__ void k_histogram(const float* __restrict__ pts, int64_t npts, BinGrid b, unsigned* __restrict__ counts) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < npts; q += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&counts[bin_of(pts + q * b.d, b)], 1u);
}

template <typename T>
__global__ void k_hist_norm(const unsigned* __restrict__ counts, int64_t nb, double npts, T* __restrict__ p) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = (T)((double)counts[i] / npts);
}

struct PointsOf {
  int kind, d;  // UOT_GEOM_GRID: axes and shape; UOT_GEOM_POINTS: row-major points
  int shape[UOT_MAX_DIM];
  const void* axes[UOT_MAX_DIM];
  const void* pts;
};

template <typename T>
__device__ __forceinline__ T coord_of(const PointsOf& P, int64_t j, int k) {
  if (P.kind == UOT_GEOM_POINTS) return reinterpret_cast<const T*>(P.pts)[j * P.d + k];
  int64_t r = j;
  for (int a = P.d - 1; a > k; --a) r /= P.shape[a];
  return reinterpret_cast<const T*>(P.axes[k])[r % P.shape[k]];
}

// F[j][0..d-1] = coordinates of point j, F[j][d] = 1.
template <typename T>
__global__ void k_coords1(PointsOf P, int64_t m, T* __restrict__ F) {
  const int c = P.d + 1;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m * c; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = q / c;
    const int k = (int)(q - j * c);
    F[q] = (k == P.d) ? T(1) : coord_of<T>(P, j, k);
  }
}

// T_i = RF[i][0..d-1] / RF[i][d]; rows of zero plan mass keep their own point.
template <typename T>
__global__ void k_bary_divide(const T* __restrict__ RF, PointsOf X, int64_t n, T* __restrict__ Tm) {
  const int d = X.d, c = d + 1;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n * d; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / d;
    const int k = (int)(q - i * d);
    const T den = RF[i * c + d];
    Tm[q] = (den > T(0)) ? RF[i * c + k] / den : coord_of<T>(X, i, k);
  }
}

template <typename T>
__global__ void k_apply_bin_map(const float* __restrict__ pts, int64_t npts, BinGrid b, const T* __restrict__ Tm,
                                float* __restrict__ out) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < npts; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t bin = bin_of(pts + q * b.d, b);
    for (int c = 0; c < b.d; ++c) out[q * b.d + c] = (float)Tm[bin * b.d + c];
  }
}

uot_status bin_grid(int d, const int* shape, BinGrid& b, int64_t& nb) {
  if (d < 1 || d > kMaxBinDim || !shape) return UOT_EINVAL;
  b.d = d;
  nb = 1;
  for (int a = 0; a < d; ++a) {
    if (shape[a] < 1) return UOT_EINVAL;
    b.shape[a] = shape[a];
    nb *= shape[a];
    if (nb > ((int64_t)1 << 31)) return UOT_EINVAL;
  }
  return UOT_OK;
}

}  // namespace

void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

namespace {
std::mutex g_smem_mu;
std::map<std::pair<int, const void*>, size_t> g_smem_limit;  // (device, kernel) -> limit set
}  // namespace

cudaError_t smem_limit_at_least(const void* kernel, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_smem_mu);
  auto it = g_smem_limit.find({dev, kernel});
  if (it == g_smem_limit.end()) {
    // the limit in force (by default 48 KB less the kernel's static shared memory)
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, kernel)) != cudaSuccess) return e;
    it = g_smem_limit.emplace(std::make_pair(dev, kernel), (size_t)fa.maxDynamicSharedSizeBytes).first;
  }
  size_t& cur = it->second;
  if (bytes <= cur) return cudaSuccess;
  if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)) != cudaSuccess)
    return e;
  cur = bytes;
  return cudaSuccess;
}

void prof_mark_begin(int family, cudaStream_t s) {
  if (!g_prof.on) return;
  std::lock_guard<std::mutex> lk(g_prof.mu);
  cudaEvent_t e = prof_event();
  cudaEventRecord(e, s);
  g_prof.pending[family] = e;
}

void prof_mark_end(int family, cudaStream_t s) {
  if (!g_prof.on) return;
  std::lock_guard<std::mutex> lk(g_prof.mu);
  cudaEvent_t e = prof_event();
  cudaEventRecord(e, s);
  g_prof.marks[family].push_back({g_prof.pending[family], e});
}

}  // namespace uot

using namespace uot;

extern "C" {

const char* uot_version(void) { return "uot-gb300 0.1 (sm_103a)"; }

const char* uot_last_error(void) { return g_last_error.c_str(); }

long long uot_launch_count(void) { return g_launches.load(); }

int uot_set_autotune(int mode) { return grid_set_autotune(mode); }

uot_status uot_force_grid_tile(int idx) { return grid_force_tile(idx) == 0 ? UOT_OK : UOT_EINVAL; }

int uot_grid_tile_count(void) { return grid_tile_count(); }

int uot_force_precise_passes(int on) { return grid_force_precise(on); }

int uot_fuse_short_passes(int on) { return grid_fuse_short_pairs(on ? 1 : 0); }

uot_status uot_selftest_bounded_wait(double seconds, void* stream) {
  clear_stale_error();
  if (!(seconds > 0.0) || seconds > 10.0) return UOT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s);
  sc.reserve<unsigned>(1);
  sc.reserve<int>(1);
  UOT_CK(sc.allocate());
  unsigned* flag = sc.take<unsigned>(1);
  int* status = sc.take<int>(1);
  UOT_SCRATCH_OK(sc);
  UOT_CK(cudaMemsetAsync(flag, 0, sizeof(unsigned), s));
  UOT_CK(cudaMemsetAsync(status, 0, sizeof(int), s));
  UOT_CK(launch_wait_selftest(flag, (unsigned long long)(seconds * 1e9), status, s));
  int h = 0;
  UOT_CK(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
  UOT_CK(cudaStreamSynchronize(s));
  if (h) {
    g_last_error = "bounded device wait expired (self-test: the flag is never set)";
    return UOT_TIMEOUT;
  }
  return UOT_OK;
}

uot_status uot_force_batch_warps(int warps) { return batch_force_warps(warps) == 0 ? UOT_OK : UOT_EINVAL; }

int uot_autotune_table(char* buf, int len) {
  const std::string t = grid_tile_table() + batch_tune_table();
  if (buf && len > 0) {
    const size_t n = std::min((size_t)(len - 1), t.size());
    memcpy(buf, t.data(), n);
    buf[n] = 0;
  }
  return (int)t.size();
}

void uot_profile_begin(void) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  for (auto& v : g_prof.marks) {
    for (auto& pr : v) {
      g_prof.pool.push_back(pr.first);
      g_prof.pool.push_back(pr.second);
    }
    v.clear();
  }
  g_prof.on = true;
}

uot_status uot_profile_end(int family, double* total_ms, long long* launches) {
  if (family < 0 || family >= PROF_NFAM || !total_ms || !launches) return UOT_EINVAL;
  std::lock_guard<std::mutex> lk(g_prof.mu);
  g_prof.on = false;
  double tot = 0.0;
  for (auto& pr : g_prof.marks[family]) {
    cudaError_t e = cudaEventSynchronize(pr.second);
    if (e != cudaSuccess) return fail_cuda(e);
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, pr.first, pr.second);
    if (e != cudaSuccess) return fail_cuda(e);
    tot += ms;
  }
  *total_ms = tot;
  *launches = (long long)g_prof.marks[family].size();
  return UOT_OK;
}

uot_status uot_histogram(const float* pts, long long npts, int d, const int* shape, int precision, void* p,
                         void* stream) {
  clear_stale_error();
  BinGrid b;
  int64_t nb = 0;
  uot_status st = bin_grid(d, shape, b, nb);
  if (st != UOT_OK) return st;
  if (!pts || !p || npts < 1 || (precision != UOT_F64 && precision != UOT_F32)) return UOT_EINVAL;
  if (npts > 0xffffffffLL) return UOT_EINVAL;  // 32-bit counters
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s);
  sc.reserve<unsigned>(nb);
  UOT_CK(sc.allocate());
  unsigned* counts = sc.take<unsigned>(nb);
  UOT_SCRATCH_OK(sc);
  UOT_CK(cudaMemsetAsync(counts, 0, nb * sizeof(unsigned), s));
  count_launches(2);
  k_histogram<<<nblocks(npts), kNT, 0, s>>>(pts, npts, b, counts);
  if (precision == UOT_F64)
    k_hist_norm<double><<<nblocks(nb), kNT, 0, s>>>(counts, nb, (double)npts, (double*)p);
  else
    k_hist_norm<float><<<nblocks(nb), kNT, 0, s>>>(counts, nb, (double)npts, (float*)p);
  UOT_CK(cudaGetLastError());
  return UOT_OK;
}

uot_status uot_barycentric_map(const uot_geom* g, const void* U, const void* V, double eps, const void* dx,
                               const void* dy, int precision, void* T, void* stream) {
  clear_stale_error();
  uot_status st = check_geom(g);
  if (st != UOT_OK) return st;
  if (!U || !V || !dx || !dy || !T || !(eps > 0.0) || (precision != UOT_F64 && precision != UOT_F32))
    return UOT_EINVAL;
  if (g->kind == UOT_GEOM_DENSE) return UOT_EUNSUPPORTED;
  const int d = (g->kind == UOT_GEOM_GRID) ? g->ndim : g->d;
  if (d + 1 > 64) return UOT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = g->n, m = g->m;
  const size_t esz = precision == UOT_F64 ? 8 : 4;
  PointsOf X, Y;
  memset(&X, 0, sizeof(X));
  memset(&Y, 0, sizeof(Y));
  X.kind = Y.kind = g->kind;
  X.d = Y.d = d;
  if (g->kind == UOT_GEOM_GRID) {
    for (int k = 0; k < d; ++k) {
      X.shape[k] = g->shape_x[k];
      X.axes[k] = g->axes_x[k];
      Y.shape[k] = g->shape_y[k];
      Y.axes[k] = g->axes_y[k];
    }
  } else {
    X.pts = g->x;
    Y.pts = g->y;
  }
  Scratch sc(s);
  sc.reserve<char>((size_t)m * (d + 1) * esz);
  sc.reserve<char>((size_t)n * (d + 1) * esz);
  UOT_CK(sc.allocate());
  char* F = sc.take<char>((size_t)m * (d + 1) * esz);
  char* RF = sc.take<char>((size_t)n * (d + 1) * esz);
  UOT_SCRATCH_OK(sc);
  count_launches(1);
  if (precision == UOT_F64)
    k_coords1<double><<<nblocks(m * (d + 1)), kNT, 0, s>>>(Y, m, (double*)F);
  else
    k_coords1<float><<<nblocks(m * (d + 1)), kNT, 0, s>>>(Y, m, (float*)F);
  UOT_CK(cudaGetLastError());
  // R (dy y) and R dy in one pass of d + 1 columns
  st = uot_apply_plan(g, U, V, eps, dx, dy, F, d + 1, 0, precision, RF, stream);
  if (st != UOT_OK) return st;
  count_launches(1);
  if (precision == UOT_F64)
    k_bary_divide<double><<<nblocks(n * d), kNT, 0, s>>>((const double*)RF, X, n, (double*)T);
  else
    k_bary_divide<float><<<nblocks(n * d), kNT, 0, s>>>((const float*)RF, X, n, (float*)T);
  UOT_CK(cudaGetLastError());
  return UOT_OK;
}

uot_status uot_apply_bin_map(const float* pts, long long npts, int d, const int* shape, const void* T,
                             int precision, float* out, void* stream) {
  clear_stale_error();
  BinGrid b;
  int64_t nb = 0;
  uot_status st = bin_grid(d, shape, b, nb);
  if (st != UOT_OK) return st;
  if (!pts || !T || !out || npts < 1 || (precision != UOT_F64 && precision != UOT_F32)) return UOT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  count_launches(1);
  if (precision == UOT_F64)
    k_apply_bin_map<double><<<nblocks(npts), kNT, 0, s>>>(pts, npts, b, (const double*)T, out);
  else
    k_apply_bin_map<float><<<nblocks(npts), kNT, 0, s>>>(pts, npts, b, (const float*)T, out);
  UOT_CK(cudaGetLastError());
  return UOT_OK;
}

uot_status uot_gibbs_log(const uot_geom* g, const void* W, const void* w, double eps,
                         int transpose, int precision, void* out, void* stream) {
  clear_stale_error();
  uot_status st = check_geom(g);
  if (st != UOT_OK) return st;
  if (!W || !w || !out || !(eps > 0.0) || !prec_ok(precision)) return UOT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nin = transpose ? g->n : g->m, nout = transpose ? g->m : g->n;
  Scratch sc(s);
  Gibbs G;
  G.g = *g;
  G.prec = precision;
  G.plan(sc, 1);
  sc.reserve<double>(nin);
  sc.reserve<double>(nin);
  sc.reserve<double>(nout);
  UOT_CK(sc.allocate());
  UOT_CK(G.take(sc, s));
  double* Wd = sc.take<double>(nin);
  double* logw = sc.take<double>(nin);
  double* od = sc.take<double>(nout);
  UOT_SCRATCH_OK(sc);
  UOT_CK(to_f64(precision, W, nin, Wd, s));
  UOT_CK(to_log(precision, w, nin, logw, s));
  Epilogue e;
  memset(&e, 0, sizeof(e));
  e.mode = EPI_SCALE;
  set_eps(e, eps);
  e.out = od;
  UOT_CK(G.apply(transpose ? 1 : 0, Wd, logw, eps, e, s));
  UOT_CK(from_f64(precision, od, nout, out, s));
  if (precision == UOT_MIXED && G.tc_err) {
    // the tensor-core pass's bounded waits report through this flag
    int htc = 0;
    UOT_CK(cudaMemcpyAsync(&htc, G.tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    UOT_CK(cudaStreamSynchronize(s));
    if (htc) {
      g_last_error = "uot_gibbs_log: a bounded wait of the tensor-core pass expired";
      return UOT_TIMEOUT;
    }
  }
  return UOT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// No-allocation variant of uot_gibbs_log.
//
// Some callers cannot allocate device memory at all: code running inside a
// CUDA stream capture that must not add allocation nodes, processes whose
// device memory is fully owned by another allocator, or real-time loops where
// an allocation can block.  For them the operator's scratch lives in one
// file-scope device array of fixed size that every GPU loading this library
// holds until the process exits.  In host code the array's name is only a
// host-side stand-in, so its device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and passed to the kernels.
// ---------------------------------------------------------------------------
namespace uot {
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)UOT_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
char* g_noalloc_addr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on the current device (set up on the
// first call per device).
cudaError_t noalloc_scratch(char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = (char*)p;
  }
  *out = g_noalloc_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace uot

extern "C" {

uot_status uot_gibbs_log_noalloc(const uot_geom* g, const void* W, const void* w, double eps,
                                 int transpose, int precision, void* out, void* stream) {
  clear_stale_error();
  // no tuning here: the tuner allocates its scratch inputs
  struct TuneHold {
    TuneHold() { grid_tune_hold(1); }
    ~TuneHold() { grid_tune_hold(0); }
  } hold;
  uot_status st = check_geom(g);
  if (st != UOT_OK) return st;
  if (!W || !w || !out || !(eps > 0.0) || !prec_ok(precision)) return UOT_EINVAL;
  if (g->kind == UOT_GEOM_DENSE) {
    g_last_error = "uot_gibbs_log_noalloc: dense cost matrices are not supported (grid and points only)";
    return UOT_EUNSUPPORTED;
  }
  if (precision == UOT_MIXED) {
    // its set-up copies the grid axes to the host and synchronises the stream
    g_last_error = "uot_gibbs_log_noalloc: UOT_MIXED is not supported (UOT_F64 and UOT_F32 only)";
    return UOT_EUNSUPPORTED;
  }
  cudaStream_t s = (cudaStream_t)stream;
  char* base = nullptr;
  UOT_CK(noalloc_scratch(&base));
  const int64_t nin = transpose ? g->n : g->m, nout = transpose ? g->m : g->n;
  Scratch sc(s, base, kNoAllocScratchBytes);
  Gibbs G;
  G.g = *g;
  G.prec = precision;
  G.host_setup = false;  // no read-back of the axes (it would synchronise the stream)
  G.plan(sc, 1);
  sc.reserve<double>(nin);
  sc.reserve<double>(nin);
  sc.reserve<double>(nout);
  if (sc.needed() > kNoAllocScratchBytes) {
    g_last_error = "uot_gibbs_log_noalloc: problem needs " + std::to_string(sc.needed()) +
                   " bytes of scratch, more than the fixed " +
                   std::to_string(kNoAllocScratchBytes) + " bytes (UOT_NOALLOC_SCRATCH_BYTES)";
    return UOT_EINVAL;
  }
  UOT_CK(sc.allocate());
  UOT_CK(G.take(sc, s));
  double* Wd = sc.take<double>(nin);
  double* logw = sc.take<double>(nin);
  double* od = sc.take<double>(nout);
  UOT_SCRATCH_OK(sc);
  // Every buffer carved here is fully written before it is read, so nothing
  // left by an earlier call needs clearing.
  UOT_CK(to_f64(precision, W, nin, Wd, s));
  UOT_CK(to_log(precision, w, nin, logw, s));
  Epilogue e;
  memset(&e, 0, sizeof(e));
  e.mode = EPI_SCALE;
  set_eps(e, eps);
  e.out = od;
  UOT_CK(G.apply(transpose ? 1 : 0, Wd, logw, eps, e, s));
  UOT_CK(from_f64(precision, od, nout, out, s));
  return UOT_OK;
}

uot_status uot_apply_plan(const uot_geom* g, const void* U, const void* V, double eps,
                          const void* dx, const void* dy, const void* f, int ncols,
                          int transpose, int precision, void* out, void* stream) {
  clear_stale_error();
  uot_status st = check_geom(g);
  if (st != UOT_OK) return st;
  if (!U || !V || !dx || !dy || !out || !(eps > 0.0) || !prec_ok(precision)) return UOT_EINVAL;
  if (ncols < 1 || ncols > 64) return UOT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = g->n, m = g->m;
  const int64_t nin = transpose ? n : m, nout = transpose ? m : n;
  Scratch sc(s);
  Gibbs G;
  G.g = *g;
  G.prec = precision;
  G.plan(sc, 1);
  for (int k = 0; k < 3; ++k) sc.reserve<double>(nin);
  sc.reserve<double>(nout);
  sc.reserve<double>(nout * ncols);
  UOT_CK(sc.allocate());
  UOT_CK(G.take(sc, s));
  double* Win = sc.take<double>(nin);
  double* W = sc.take<double>(nin);
  double* logw = sc.take<double>(nin);
  double* Sh = sc.take<double>(nout);
  double* od = sc.take<double>(nout * ncols);
  UOT_SCRATCH_OK(sc);
  UOT_CK(to_f64(precision, transpose ? U : V, nin, Win, s));
  UOT_CK(to_f64(precision, transpose ? V : U, nout, Sh, s));
  UOT_CK(to_log(precision, transpose ? dx : dy, nin, logw, s));
  for (int c = 0; c < ncols; ++c) {
    count_launches(1);
    if (precision == UOT_F64)
      k_add_logf<double><<<nblocks(nin), kNT, 0, s>>>(Win, (const double*)f, ncols, c, nin, eps, W);
    else
      k_add_logf_ff<<<nblocks(nin), kNT, 0, s>>>(Win, (const float*)f, ncols, c, nin, eps, W);
    UOT_CK(cudaGetLastError());
    Epilogue e;
    memset(&e, 0, sizeof(e));
    e.mode = EPI_PLAN;
    set_eps(e, eps);
    e.out = od;
    e.pot_shift = Sh;
    e.ncols = ncols;
    e.col = c;
    UOT_CK(G.apply(transpose ? 1 : 0, W, logw, eps, e, s));
  }
  UOT_CK(from_f64(precision, od, nout * ncols, out, s));
  return UOT_OK;
}

uot_status uot_objective(const uot_geom* g, const void* p, const void* dx, const void* q,
                         const void* dy, const uot_div* F1, const uot_div* F2, double eps,
                         const void* U, const void* V, int precision, double* out, void* stream) {
  clear_stale_error();
  uot_status st = check_geom(g);
  if (st != UOT_OK) return st;
  if (!p || !dx || !q || !dy || !U || !V || !out || !(eps > 0.0) || !prec_ok(precision) ||
      !div_ok(F1) || !div_ok(F2))
    return UOT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = g->n, m = g->m;
  Scratch sc(s);
  Gibbs G;
  G.g = *g;
  G.prec = precision;
  G.plan(sc, 1);
  for (int k = 0; k < 6; ++k) sc.reserve<double>(n);  // Ud logp logdx r1 zK1 S1
  for (int k = 0; k < 4; ++k) sc.reserve<double>(m);  // Vd logq logdy r2
  sc.reserve<double>(n > m ? n : m);                  // zero
  sc.reserve<double>(16);                             // acc
  UOT_CK(sc.allocate());
  UOT_CK(G.take(sc, s));
  double* Ud = sc.take<double>(n);
  double* Vd = sc.take<double>(m);
  double* logp = sc.take<double>(n);
  double* logq = sc.take<double>(m);
  double* logdx = sc.take<double>(n);
  double* logdy = sc.take<double>(m);
  double* r1 = sc.take<double>(n);
  double* r2 = sc.take<double>(m);
  double* zK1 = sc.take<double>(n);
  double* S1 = sc.take<double>(n);
  double* zero = sc.take<double>(n > m ? n : m);
  double* acc = sc.take<double>(16);
  UOT_SCRATCH_OK(sc);
  UOT_CK(to_f64(precision, U, n, Ud, s));
  UOT_CK(to_f64(precision, V, m, Vd, s));
  UOT_CK(to_log(precision, p, n, logp, s));
  UOT_CK(to_log(precision, q, m, logq, s));
  UOT_CK(to_log(precision, dx, n, logdx, s));
  UOT_CK(to_log(precision, dy, m, logdy, s));
  count_launches(1);
  k_fill<<<nblocks(n > m ? n : m), kNT, 0, s>>>(zero, n > m ? n : m, 0.0);
  UOT_CK(cudaMemsetAsync(acc, 0, 16 * 8, s));
  Epilogue e;
  memset(&e, 0, sizeof(e));
  set_eps(e, eps);
  // r1 = R dy, r2 = R^T dx
  e.mode = EPI_PLAN;
  e.ncols = 1;
  e.out = r1;
  e.pot_shift = Ud;
  UOT_CK(G.apply(0, Vd, logdy, eps, e, s));
  e.out = r2;
  e.pot_shift = Vd;
  UOT_CK(G.apply(1, Ud, logdx, eps, e, s));
  // z_i = log sum_j K_ij dy_j  (for sum dx dy K) and S = eps log K(b.dy)
  e.mode = EPI_RAW;
  e.out = zK1;
  UOT_CK(G.apply(0, zero, logdy, eps, e, s));
  e.mode = EPI_SCALE;
  e.out = S1;
  UOT_CK(G.apply(0, Vd, logdy, eps, e, s));
  const DivParams D1 = make_div(*F1), D2 = make_div(*F2);
  if (precision != UOT_F64) {
    double* arrs_n[] = {Ud, logp, logdx, r1, zK1, S1};
    double* arrs_m[] = {Vd, logq, logdy, r2};
    for (double* a : arrs_n) {
      count_launches(1);
      k_ff_to_double<<<nblocks(n), kNT, 0, s>>>(a, n);
    }
    for (double* a : arrs_m) {
      count_launches(1);
      k_ff_to_double<<<nblocks(m), kNT, 0, s>>>(a, m);
    }
    UOT_CK(cudaGetLastError());
  }
  count_launches(1);
  k_objective_side<<<nblocks(n) > 1024 ? 1024 : nblocks(n), kNT, 0, s>>>(r1, Ud, logp, logdx, zK1, S1, D1, eps, n, acc);
  count_launches(1);
  k_objective_side<<<nblocks(m) > 1024 ? 1024 : nblocks(m), kNT, 0, s>>>(r2, Vd, logq, logdy, nullptr, nullptr, D2, eps, m, acc + 8);
  UOT_CK(cudaGetLastError());
  double h[16];
  UOT_CK(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
  UOT_CK(cudaStreamSynchronize(s));
  // eps sum dx dy (R - K) = eps (sum dx r1 - sum dx dy K)
  const double mass_term = eps * (h[3] - h[4]);
  const double primal = h[0] + h[8] + h[2] + h[10] - mass_term;
  const double dual = -h[1] - h[9] - mass_term;
  out[0] = primal;
  out[1] = dual;
  out[2] = (h[0] + h[1] + h[2]) + (h[8] + h[9] + h[10]);
  out[3] = (h[6] > 0.0) ? h[5] / h[6] : 0.0;
  return UOT_OK;
}

}  // extern "C"
