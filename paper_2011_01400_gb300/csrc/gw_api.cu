// C ABI of the G0W0 hot path: plan creation and the per-q calls (see include/gw.h).
#include "gw_internal.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

namespace gw {
std::atomic<unsigned long long> g_launch_count{0};
std::atomic<unsigned long long> g_alloc_count{0};
}

using namespace gw;

namespace {

thread_local std::string g_last_error;

gw_status fail(gw_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

}  // namespace

namespace gw {
void gw_set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace gw

namespace {

#define GW_CUDA(call)                                                                                  \
  do {                                                                                                 \
    cudaError_t e_ = (call);                                                                           \
    if (e_ != cudaSuccess) {                                                                           \
      return fail(GW_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));                     \
    }                                                                                                  \
  } while (0)

// Gauss-Legendre nodes and weights on (-1, 1) by Newton's method on P_n (ascending nodes).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int l = 2; l <= n; ++l) {
        double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
        p0 = p1;
        p1 = p2;
      }
      double pn = (n == 1) ? z : p1;
      double pm = (n == 1) ? 1.0 : p0;
      dp = n * (z * pn - pm) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int l = 2; l <= n; ++l) {
        double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
        p0 = p1;
        p1 = p2;
      }
      double pn = (n == 1) ? z : p1, pm = (n == 1) ? 1.0 : p0;
      dp = n * (z * pn - pm) / (z * z - 1.0);
    }
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

template <typename T> struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
};

__global__ void k_frob_scale(int N, const c128* V, long long s, double* out) {
  __shared__ double red[256];
  const c128* a = V + blockIdx.x * s;
  double acc = 0;
  for (long long e = threadIdx.x; e < (long long)N * N; e += blockDim.x) acc += a[e].re * a[e].re + a[e].im * a[e].im;
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int t = blockDim.x / 2; t > 0; t >>= 1) {
    if (threadIdx.x < t) red[threadIdx.x] += red[threadIdx.x + t];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sqrt(red[0]);
}

// Time-reversal check of the inputs: out[0] = max |eps_n(k) - eps_n(-k)|, out[1] = max |eps|,
// out[2] = max |V(q) - conj(V(-q))|, out[3] = max |V| (as the bits of non-negative doubles).
__global__ void k_trs_check(int n1, int n2, int n3, int NBd, const double* __restrict__ eps, int N,
                            const c128* __restrict__ V, unsigned long long* out) {
  const int NK = n1 * n2 * n3;
  const long long NN = (long long)N * N;
  double de = 0, ae = 0, dv = 0, av = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)NK * NBd;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e / NBd), n = (int)(e % NBd);
    const int i3 = k % n3, i2 = (k / n3) % n2, i1 = k / (n2 * n3);
    const int mk = (((n1 - i1) % n1) * n2 + (n2 - i2) % n2) * n3 + (n3 - i3) % n3;
    de = fmax(de, fabs(eps[e] - eps[(long long)mk * NBd + n]));
    ae = fmax(ae, fabs(eps[e]));
  }
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)NK * NN;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e / NN);
    const long long r = e % NN;
    const int i3 = k % n3, i2 = (k / n3) % n2, i1 = k / (n2 * n3);
    const int mk = (((n1 - i1) % n1) * n2 + (n2 - i2) % n2) * n3 + (n3 - i3) % n3;
    const c128 a = V[e], b = V[(long long)mk * NN + r];
    dv = fmax(dv, fmax(fabs(a.re - b.re), fabs(a.im + b.im)));
    av = fmax(av, fmax(fabs(a.re), fabs(a.im)));
  }
  atomicMax(out, (unsigned long long)__double_as_longlong(de));
  atomicMax(out + 1, (unsigned long long)__double_as_longlong(ae));
  atomicMax(out + 2, (unsigned long long)__double_as_longlong(dv));
  atomicMax(out + 3, (unsigned long long)__double_as_longlong(av));
}

// Y = V / c (typed), Z = I
template <typename T>
__global__ void k_ns_init(int N, const c128* V, long long s, const double* c, cplx<T>* Y, cplx<T>* Z) {
  const int b = blockIdx.y;
  const double inv = 1.0 / c[b];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)N * N;
       e += (long long)gridDim.x * blockDim.x) {
    c128 v = V[b * s + e];
    Y[b * s + e] = cplx<T>{(T)(v.re * inv), (T)(v.im * inv)};
    int i = (int)(e / N), j = (int)(e % N);
    Z[b * s + e] = cplx<T>{(T)(i == j ? 1 : 0), (T)0};
  }
}
// out = sqrt(c) * Y (c128)
template <typename T>
__global__ void k_ns_final(int N, const cplx<T>* Y, long long s, const double* c, c128* out) {
  const int b = blockIdx.y;
  const double f = sqrt(c[b]);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)N * N;
       e += (long long)gridDim.x * blockDim.x) {
    cplx<T> y = Y[b * s + e];
    out[b * s + e] = c128{f * (double)y.re, f * (double)y.im};
  }
}

}  // namespace

// learned frequency surrogate attached to a plan (gw_surrogate_enable)
struct SurState {
  gw_surrogate_s* model = nullptr;
  bool on = false;
  int nc = 0, nf = 0, k = 0, nb = 0, iters = 0;
  std::vector<int> coarse, fine;
  int* d_jmap = nullptr;       // [nw]: coarse position, or -(fine position + 1)
  int *d_cidx = nullptr, *d_fidx = nullptr;  // grid indices of the coarse [nc] and fine [nf] frequencies
  double* d_freq_c = nullptr;  // [nc]
  c128* d_start = nullptr;     // [N][nb]
  int bcap = 0;                // problems the batch buffers below hold
  c128 *d_Y = nullptr, *d_Q = nullptr, *d_T = nullptr;               // [bcap][N][nb]
  c128 *d_G = nullptr, *d_Linv = nullptr, *d_H = nullptr, *d_Z = nullptr;  // [bcap][nb][nb]
  double* d_theta = nullptr;   // [bcap][nb]
  // training-data pass (gw_surrogate_data): per group of the full-grid q loop
  c128 *g_Af = nullptr, *g_Uf = nullptr;  // [qb][N][N], [qb][N][k]
  float* d_df = nullptr;                  // [qb * k][nw]
  c128* d_A1 = nullptr;        // [N][N] eps~(w_ref) - 1 of gw_surrogate_modes
  c128* d_U1 = nullptr;        // [N][k]
  c128* d_XU = nullptr;        // [max(nw, nc)][N][k]
  c128* d_B = nullptr;         // [N][k] V^1/2 U (c128, or c64 in its first half)
  void* d_P = nullptr;         // [sig_rows][k] projections (c64 or c128)
  float* d_Sc = nullptr;       // [sig_rows][nc]
  double* d_Sc_d = nullptr;    // [sig_rows][nc]
  // q-group buffers of the surrogate pass
  int qbs = 0;
  c128 *g_chi0 = nullptr, *g_E = nullptr, *g_work = nullptr, *g_A = nullptr, *g_U = nullptr;
  float *d_d = nullptr, *d_x = nullptr, *d_sig = nullptr, *d_g = nullptr, *d_coef = nullptr;
};

// Autotuner of the fp32 shared-memory M kernels. Per device and call shape (kernel, na, nb) both
// thread mappings are run at first use on the calling plan's stream -- one warm-up launch, then one
// timed launch each (CUDA events) -- and the faster one is recorded process-wide for every later
// call of that shape. The two mappings write bit-identical rows, so the repeated launches only cost
// time; results never depend on the choice.
struct MgenTuner {
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  static std::map<std::array<int, 4>, int>& table() {
    static std::map<std::array<int, 4>, int> t;
    return t;
  }
  static std::mutex& table_mutex() {
    static std::mutex m;
    return m;
  }
  ~MgenTuner() {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
  }
  // launch(variant) issues the kernel on st; returns false on a CUDA error
  template <typename F> bool run(int kind, int na, int nb, cudaStream_t st, F&& launch) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    const std::array<int, 4> key{dev, kind, na, nb};
    {
      std::lock_guard<std::mutex> lk(table_mutex());
      auto it = table().find(key);
      if (it != table().end()) {
        const int v = it->second;
        launch(v);
        return true;
      }
    }
    for (cudaEvent_t& e : ev)
      if (!e && cudaEventCreate(&e) != cudaSuccess) return false;
    launch(0);
    if (cudaEventRecord(ev[0], st) != cudaSuccess) return false;
    launch(0);
    if (cudaEventRecord(ev[1], st) != cudaSuccess) return false;
    launch(1);
    if (cudaEventRecord(ev[2], st) != cudaSuccess || cudaEventSynchronize(ev[2]) != cudaSuccess) return false;
    float t0 = 0.f, t1 = 0.f;
    if (cudaEventElapsedTime(&t0, ev[0], ev[1]) != cudaSuccess || cudaEventElapsedTime(&t1, ev[1], ev[2]) != cudaSuccess)
      return false;
    std::lock_guard<std::mutex> lk(table_mutex());
    table()[key] = (t1 < t0) ? 1 : 0;
    return true;
  }
};

struct gw_plan_s {
  gw_problem p{};
  gw_precision prec;
  bool fp64;
  cudaStream_t st = nullptr;
  int NK, N, NB, NBd, nocc, nunocc, nsig, nw, natoms;
  std::vector<int> basis_atom, aux_atom, R;
  LriGeom geom{};
  std::vector<double> freq, fweight;
  double mu = 0.0;
  int err = 0;              // sticky error
  int chi0_q = -1, wc_q = -1;
  // device memory owned by the plan
  std::vector<void*> allocs;
  std::vector<size_t> alloc_bytes;  // size of each entry of allocs
  size_t ws_bytes = 0;              // sum of alloc_bytes
  size_t ws_limit = 0;              // GW_WORKSPACE_LIMIT (bytes; 0 = no limit)
  int dev = -1;                     // CUDA device that was current at gw_plan_create
  bool trs = false;                 // time-reversal symmetric inputs (gw_problem.time_reversal)
  // time reversal without a q -> 0 direction: Sigma_c(-k) = Sigma_c(k), so gw_g0w0 computes the
  // target k with k <= -k only (d_ktab, n_krep) into d_sigtmp and fills the others from them
  int* d_ktab = nullptr;
  int* d_isrep = nullptr;
  int n_krep = 0;
  c128* d_sigtmp = nullptr;
  double *d_freq = nullptr, *d_fw = nullptr, *d_mu = nullptr;
  void* d_T1 = nullptr;     // c128 (FP64) or c64 (split)
  c128* d_Vh = nullptr;     // [NK][N][N] V(q)^1/2 (full, truncated at q=0)
  c128* d_Vb0 = nullptr;    // [N][N] V(0)^1/2 without the lambda=1 component
  c128* d_x1 = nullptr;     // [N]
  double* d_v1 = nullptr;
  double h_v1 = 0.0;
  c128* d_chi0 = nullptr;   // [nw][N][N]
  c128* d_E = nullptr;      // [nw][N][N] eps~ then eps~^-1 - 1
  c128* d_Wc = nullptr;     // [nw][N][N]
  c128* d_work = nullptr;   // [nw][N][N]
  c128* d_tmp = nullptr;    // [nw][N][N]
  c128* d_sigma = nullptr;  // [NK][nsig][nw]
  double* d_head = nullptr; // [nw]
  c128* d_h = nullptr;      // [nw][N]
  // direction-averaged q = 0 (head_wings = 2)
  c128* d_pq3 = nullptr;    // [3][ldm] Cartesian components of p . q^
  double* d_A6 = nullptr;   // [nw][6] head tensor
  c128 *d_h3 = nullptr, *d_Y3 = nullptr, *d_G3 = nullptr;  // [nw][3][N] wings, y_a; [nw][N][3] g_a
  double* d_m10 = nullptr;  // [nw][10] direction moments of the Schur complement
  double* d_dirs = nullptr; // [n_dirs][4] direction rule (x, y, z, weight)
  int n_dirs = 0;
  int* d_status = nullptr;
  // chunk workspaces
  int chi_nkk = 1, sig_nkk = 1;
  void* d_M = nullptr;        // chi0 M [N][ldm] (c128 or c64)
  long long ldm = 0;
  double* d_delta = nullptr;  // [ldm]
  float* d_delta_f = nullptr;
  c128* d_pq = nullptr;       // [ldm]
  void* d_A = nullptr;        // sigma rows [R][N]
  void* d_Apl[2] = {};        // split precision: bf16 / tf32 pieces of the sigma rows [R][2*Kx]
  double* d_Sx = nullptr;     // gw_sigma_x: S per row; FP32 rows A V [R][Kx] and V(q) in fp32
  c64 *d_Ux = nullptr, *d_Vx32 = nullptr;
  void* d_U = nullptr;        // [R][N]
  double* d_S_d = nullptr;    // [R][nw]
  float* d_S_f = nullptr;
  long long sig_rows = 0;
  float* d_Praw = nullptr;    // fp32 plane of M for the tensor-core chi0 [N][2*ldm]
  void* d_Pb[6] = {};         // B1 / B2 split planes [N][2*ldm]
  int n_bpl = 0;
  int seg_rows = 8192;        // pair rows per FP64 promotion segment of the tensor-core chi0 (cfg1, q = 1:
                              // 2.4e-7 relative against the FP64 path, 2.2e-7 at 2048 rows, 6% slower)
  float* d_wtab = nullptr;    // [nw][ldm] Lorentzian weights
  unsigned* d_absmax = nullptr;  // largest |re|, |im| of the chi0 M plane (float bits)
  int* d_eB = nullptr;        // FP16: exponent of the B plane scale
  double* d_escale = nullptr; // [nw] factors of the drained chi0 sums
  Chi0Plan* chi0plan = nullptr;   // work lists of the tcgen05 chi0 kernel (and the screen products)
  float* d_hb[2] = {nullptr, nullptr};  // screen products: TF32 pieces of the Hermitian right operand
  float* d_hones = nullptr;             // [Kpad] unit weights
  double* d_hesc = nullptr;             // [nw]
  // frequency compression of the split-precision chi0 (k_compress.cu)
  // largest relative residual |W_j - sum_{t<T} E_jt v_t| / |W_j| over the frequencies j that the
  // compression may leave (computed in FP64 over all pair rows); 0 disables. 3e-8 is below the
  // fp32 rounding of the weights themselves
  double compress_tol = 3e-8;
  c128 *d_wG = nullptr, *d_wU = nullptr, *d_C = nullptr;  // [NK][nw][nw], [NK][nw][nw], [nw][N][N]
  double* d_wlam = nullptr;   // [NK][nw]
  double *d_wn = nullptr, *d_wE = nullptr, *d_wP = nullptr, *d_werr = nullptr;  // [NK][nw], [NK][nw][nw] x2,
                                                                               // [NK][nw][nw+1]
  std::vector<int> comp_qs;   // q points (in order) whose weight spectra are ready
  int comp_nw = 0;            // grid size they were computed for
  std::vector<int> comp_T;    // components kept per q of that range
  int last_T = 0;             // components kept for the last q
  int Kx = 0;                 // n_aux rounded up to 32 (K of the Sigma contraction)
  PlaneSet d_Wpl{};           // W^c split planes [nw*N][2*Kx]
  c64* d_Vh32 = nullptr;      // FP32 copies of V^1/2 for the split-precision screen
  c64* d_Vb32 = nullptr;
  // q-group buffers of gw_g0w0
  c128 *g_chi0 = nullptr, *g_E = nullptr, *g_work = nullptr;
  int qb = 0;
  double group_budget = 8.0e9;  // bytes for the q-group buffers of gw_g0w0
  MgenTuner mtune;              // picks the thread mapping of the fp32 M kernels per call shape
  SurState sur;
  // batch plan (n_sys > 1): one plan per system, each on its own stream; the batch plan itself
  // holds no device memory
  std::vector<gw_plan_s*> subs;
  std::vector<cudaStream_t> sub_streams;
  // timing of the chi0 contraction launches of the last call (CUDA events on the plan's stream)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double last_chi0_ms = 0.0, last_chi0_flops = 0.0, chi0_flops_acc = 0.0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> evs;
  size_t ev_used = 0;
  gw_status event_pair(cudaEvent_t& a, cudaEvent_t& b) {
    if (ev_used == evs.size()) {
      cudaEvent_t x, y;
      if (cudaEventCreate(&x) != cudaSuccess || cudaEventCreate(&y) != cudaSuccess)
        return fail(GW_ERR_CUDA, "cudaEventCreate failed");
      evs.push_back({x, y});
    }
    a = evs[ev_used].first;
    b = evs[ev_used].second;
    ++ev_used;
    return GW_OK;
  }
  void reset_timing() {
    ev_used = 0;
    chi0_flops_acc = 0.0;
  }
  gw_status collect_timing() {
    double ms = 0.0;
    for (size_t i = 0; i < ev_used; ++i) {
      float t = 0.f;
      cudaError_t e = cudaEventSynchronize(evs[i].second);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, evs[i].first, evs[i].second);
      if (e != cudaSuccess) return fail(GW_ERR_CUDA, std::string("chi0 timing: ") + cudaGetErrorString(e));
      ms += t;
    }
    last_chi0_ms = ms;
    last_chi0_flops = chi0_flops_acc;
    return GW_OK;
  }
};

namespace {

template <typename T> gw_status dalloc(gw_plan_s* P, T** ptr, size_t count) {
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  if (P->ws_limit && P->ws_bytes + bytes > P->ws_limit)
    return fail(GW_ERR_NOMEM, "workspace limit GW_WORKSPACE_LIMIT = " + std::to_string(P->ws_limit) +
                                  " bytes reached: " + std::to_string(P->ws_bytes) + " held, " +
                                  std::to_string(bytes) + " more requested");
  void* p = nullptr;
  ++g_alloc_count;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(GW_ERR_NOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                                  cudaGetErrorString(e));
  }
  P->allocs.push_back(p);
  P->alloc_bytes.push_back(bytes);
  P->ws_bytes += bytes;
  *ptr = static_cast<T*>(p);
  return GW_OK;
}

// frees the most recent dalloc
void dfree_last(gw_plan_s* P) {
  cudaFree(P->allocs.back());
  P->allocs.pop_back();
  P->ws_bytes -= P->alloc_bytes.back();
  P->alloc_bytes.pop_back();
}

#define GW_TRY(x)                    \
  do {                               \
    gw_status s_ = (x);              \
    if (s_ != GW_OK) return s_;      \
  } while (0)

gw_status check_launch(gw_plan_s* P, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    P->err = 1;
    return fail(GW_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  }
  return GW_OK;
}

gw_status read_status(gw_plan_s* P, const char* where) {
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, P->d_status, sizeof(int), cudaMemcpyDeviceToHost, P->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->st);
  if (e != cudaSuccess) {
    P->err = 1;
    return fail(GW_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  }
  if (st & ST_TIMEOUT) {
    P->err = 1;
    return fail(GW_ERR_TIMEOUT, std::string(where) + ": a device-side wait exceeded its bound");
  }
  if (st & ST_NOT_PD) {
    P->err = 1;
    return fail(GW_ERR_NOT_PD, std::string(where) + ": eps~ is not positive definite (non-positive pivot)");
  }
  if (st & ST_BADARG) {
    P->err = 1;
    return fail(GW_ERR_CUDA, std::string(where) + ": a kernel bounds check failed");
  }
  return GW_OK;
}

// V^1/2 of a batch of Hermitian PD matrices by the coupled Newton-Schulz iteration
//   Y0 = V/c, Z0 = I;  T = (3 I - Z Y)/2;  Y <- Y T;  Z <- T Z;   V^1/2 = sqrt(c) Y,
// c = ||V||_F. FP64 for the FP64 method, FP32 otherwise.
template <typename T>
gw_status newton_schulz(gw_plan_s* P, const c128* V, c128* out, int batch, int iters) {
  const int N = P->N;
  const long long s = (long long)N * N;
  double* d_c;
  cplx<T> *Y, *Z, *Tm, *Y2;
  GW_TRY(dalloc(P, &d_c, batch));
  GW_TRY(dalloc(P, &Y, s * batch));
  GW_TRY(dalloc(P, &Z, s * batch));
  GW_TRY(dalloc(P, &Tm, s * batch));
  GW_TRY(dalloc(P, &Y2, s * batch));
  ++::gw::g_launch_count, k_frob_scale<<<batch, 256, 0, P->st>>>(N, V, s, d_c);
  dim3 g(std::min<long long>((s + 255) / 256, 1024), batch);
  ++::gw::g_launch_count, k_ns_init<T><<<g, 256, 0, P->st>>>(N, V, s, d_c, Y, Z);
  const cplx<T> one{(T)1, (T)0}, zero{(T)0, (T)0}, mhalf{(T)-0.5, (T)0};
  for (int it = 0; it < iters; ++it) {
    // Tm = -0.5 Z Y + 1.5 I
    launch_zgemm<T>(N, N, N, mhalf, Z, N, s, OP_N, Y, N, s, OP_N, zero, Tm, N, s, batch, P->st);
    launch_axpby_identity<T>(N, Tm, s, batch, (T)1.5, P->st);
    launch_zgemm<T>(N, N, N, one, Y, N, s, OP_N, Tm, N, s, OP_N, zero, Y2, N, s, batch, P->st);
    launch_zgemm<T>(N, N, N, one, Tm, N, s, OP_N, Z, N, s, OP_N, zero, Y, N, s, batch, P->st);  // Y <- T Z (temp)
    std::swap(Z, Y);   // Z = T Z
    std::swap(Y, Y2);  // Y = Y T
  }
  ++::gw::g_launch_count, k_ns_final<T><<<g, 256, 0, P->st>>>(N, Y, s, d_c, out);
  GW_TRY(check_launch(P, "newton_schulz"));
  cudaError_t e = cudaStreamSynchronize(P->st);
  if (e != cudaSuccess) return fail(GW_ERR_CUDA, std::string("newton_schulz: ") + cudaGetErrorString(e));
  // release the temporaries (they were the last five allocations)
  for (int i = 0; i < 5; ++i) {
    dfree_last(P);
  }
  return GW_OK;
}

gw_status herm_gemm(gw_plan_s* P, const c64* A, bool a_batch, const c128* H64, const c64* H32, bool h_batch,
                    double alpha, c128* C, int nb);

// The same iteration on the tensor cores for the split path: its three products per step as TF32
// two-piece products, FP64-accumulated, in chunks of n_freq matrices (the screen's product
// workspace). The kernel multiplies by the conjugate transpose of the rows it is given, so every
// right operand goes in as its conjugate transpose, written next to it when it is formed. (Y, Z and
// T are Hermitian in exact arithmetic, but taking H^H for H, or projecting them on their Hermitian
// parts, turns the rounding into a mode that grows after convergence; the plain products do not.)
gw_status newton_schulz_tc(gw_plan_s* P, c128* Vio, int batch, int iters) {
  const int N = P->N, nb = P->nw;
  const long long s = (long long)N * N;
  double* d_c;
  c64 *Y, *Yh, *Z, *Zh, *Tm, *Th;
  c128* C;
  GW_TRY(dalloc(P, &d_c, batch));
  GW_TRY(dalloc(P, &Y, s * nb));
  GW_TRY(dalloc(P, &Yh, s * nb));
  GW_TRY(dalloc(P, &Z, s * nb));
  GW_TRY(dalloc(P, &Zh, s * nb));
  GW_TRY(dalloc(P, &Tm, s * nb));
  GW_TRY(dalloc(P, &Th, s * nb));
  GW_TRY(dalloc(P, &C, s * nb));
  unsigned* d_dev;
  GW_TRY(dalloc(P, &d_dev, 1));
  ++::gw::g_launch_count, k_frob_scale<<<batch, 256, 0, P->st>>>(N, Vio, s, d_c);
  for (int b0 = 0; b0 < batch; b0 += nb) {
    const int n = std::min(nb, batch - b0);
    dim3 g(std::min<long long>((s + 255) / 256, 1024), n);
    ++::gw::g_launch_count, k_ns_init<float><<<g, 256, 0, P->st>>>(N, Vio + b0 * s, s, d_c + b0, Y, Z);
    // Y0 = V / c is Hermitian and Z0 = I: their conjugate transposes are themselves
    if (cudaMemcpyAsync(Yh, Y, sizeof(c64) * s * n, cudaMemcpyDeviceToDevice, P->st) != cudaSuccess ||
        cudaMemcpyAsync(Zh, Z, sizeof(c64) * s * n, cudaMemcpyDeviceToDevice, P->st) != cudaSuccess)
      return fail(GW_ERR_CUDA, "newton_schulz: copy failed");
    for (int it = 0; it < iters; ++it) {
      // T = 1.5 I - 0.5 Z Y;  Y <- Y T;  Z <- T Z
      GW_TRY(herm_gemm(P, Z, true, nullptr, Yh, true, -0.5, C, n));
      launch_take_both(N, C, s, n, 1.5f, Tm, Th, P->st);
      // converged chunk: once max |T - I| < 1e-4 the step below leaves it ~1e-8 from I (the
      // iteration converges quadratically), below the FP32 rounding of the products
      bool last = false;
      if (it >= 6 && it % 2 == 0) {
        unsigned hdev = 0;
        if (cudaMemsetAsync(d_dev, 0, sizeof(unsigned), P->st) != cudaSuccess) return fail(GW_ERR_CUDA, "newton_schulz");
        launch_dev_identity(N, Tm, s * n, d_dev, P->st);
        if (cudaMemcpyAsync(&hdev, d_dev, sizeof(unsigned), cudaMemcpyDeviceToHost, P->st) != cudaSuccess ||
            cudaStreamSynchronize(P->st) != cudaSuccess)
          return fail(GW_ERR_CUDA, "newton_schulz: convergence check failed");
        float dev;
        std::memcpy(&dev, &hdev, sizeof(float));
        last = dev < 1e-4f;
      }
      GW_TRY(herm_gemm(P, Y, true, nullptr, Th, true, 1.0, C, n));
      launch_take_both(N, C, s, n, 0.0f, Y, Yh, P->st);
      if (last) break;
      GW_TRY(herm_gemm(P, Tm, true, nullptr, Zh, true, 1.0, C, n));
      launch_take_both(N, C, s, n, 0.0f, Z, Zh, P->st);
    }
    ++::gw::g_launch_count, k_ns_final<float><<<g, 256, 0, P->st>>>(N, Y, s, d_c + b0, Vio + b0 * s);
  }
  GW_TRY(check_launch(P, "newton_schulz"));
  cudaError_t e = cudaStreamSynchronize(P->st);
  if (e != cudaSuccess) return fail(GW_ERR_CUDA, std::string("newton_schulz: ") + cudaGetErrorString(e));
  for (int i = 0; i < 9; ++i) dfree_last(P);
  return GW_OK;
}

gw_status validate(const gw_problem* p, int n_sys) {
  if (!p) return fail(GW_ERR_ARG, "problem is NULL");
  if (n_sys != 1) return fail(GW_ERR_ARG, "validate: one problem at a time");
  for (int d = 0; d < 3; ++d)
    if (p->nk[d] < 1 || p->nk[d] > 64) return fail(GW_ERR_ARG, "nk out of range [1, 64]");
  if (p->n_atoms < 1 || p->n_atoms > 64) return fail(GW_ERR_ARG, "n_atoms out of range [1, 64]");
  if (p->n_basis < 1 || p->n_bands < 2 || p->n_bands > p->n_basis) return fail(GW_ERR_ARG, "bad n_basis / n_bands");
  if (p->n_occ < 1 || p->n_occ >= p->n_bands) return fail(GW_ERR_ARG, "n_occ must be in [1, n_bands)");
  if (p->n_aux < 1 || p->n_aux > 4096) return fail(GW_ERR_ARG, "n_aux out of range [1, 4096]");
  if (!p->basis_atom || !p->aux_atom || !p->R) return fail(GW_ERR_ARG, "basis_atom / aux_atom / R is NULL");
  if (p->n_R < 1 || p->n_R > 64) return fail(GW_ERR_ARG, "n_R out of range [1, 64]");
  if (!p->eps || !p->evec || !p->ctil_R || !p->V) return fail(GW_ERR_ARG, "a device input pointer is NULL");
  if (p->head_wings < 0 || p->head_wings > 2) return fail(GW_ERR_ARG, "head_wings must be 0, 1 or 2");
  for (int d = 0; d < 3; ++d)
    if (!(std::fabs(p->k_offset[d]) <= 1.0)) return fail(GW_ERR_ARG, "k_offset components must be in [-1, 1]");
  if (p->time_reversal && (p->k_offset[0] != 0.0 || p->k_offset[1] != 0.0 || p->k_offset[2] != 0.0))
    return fail(GW_ERR_ARG, "time_reversal needs an unshifted k mesh (k_offset = 0)");
  if (p->head_wings && (!p->pmom || !(p->omega_cell > 0.0) || !std::isfinite(p->omega_cell)))
    return fail(GW_ERR_ARG, "head_wings needs pmom and omega_cell > 0");
  if (p->head_wings == 1) {
    const double q2 = p->qhat[0] * p->qhat[0] + p->qhat[1] * p->qhat[1] + p->qhat[2] * p->qhat[2];
    if (!(std::fabs(q2 - 1.0) <= 1e-9)) return fail(GW_ERR_ARG, "head_wings = 1 needs a unit vector qhat");
  }
  if (p->n_freq < 1 || p->n_freq > 256) return fail(GW_ERR_ARG, "n_freq out of range [1, 256]");
  if ((p->freq == nullptr) != (p->freq_w == nullptr)) return fail(GW_ERR_ARG, "freq and freq_w: both or neither");
  if (p->freq) {
    for (int j = 0; j < p->n_freq; ++j) {
      if (!(p->freq[j] > 0.0) || !std::isfinite(p->freq[j]) || !(p->freq_w[j] > 0.0) || !std::isfinite(p->freq_w[j]))
        return fail(GW_ERR_ARG, "freq and freq_w must be positive and finite");
      for (int i = 0; i < j; ++i)
        if (p->freq[i] == p->freq[j]) return fail(GW_ERR_ARG, "freq must be distinct");
    }
  } else if (!(p->omega0 > 0.0) || !std::isfinite(p->omega0)) {
    return fail(GW_ERR_ARG, "omega0 must be > 0");
  }
  if (p->sigma_lo < 0 || p->sigma_hi > p->n_bands || p->sigma_lo >= p->sigma_hi)
    return fail(GW_ERR_ARG, "sigma window must satisfy 0 <= lo < hi <= n_bands");
  if (!(p->spin > 0.0) || !std::isfinite(p->spin)) return fail(GW_ERR_ARG, "spin must be > 0");
  if (std::isinf(p->mu)) return fail(GW_ERR_ARG, "mu must be finite (or NaN for midgap)");
  if (p->prec != GW_FP64 && p->prec != GW_3XTF32 && p->prec != GW_3XBF16 && p->prec != GW_3XFP16)
    return fail(GW_ERR_ARG, "bad precision");
  for (int i = 0; i < p->n_basis; ++i) {
    if (p->basis_atom[i] < 0 || p->basis_atom[i] >= p->n_atoms) return fail(GW_ERR_ARG, "basis_atom out of range");
    if (i && p->basis_atom[i] < p->basis_atom[i - 1]) return fail(GW_ERR_ARG, "basis_atom must be non-decreasing");
  }
  for (int i = 0; i < p->n_aux; ++i) {
    if (p->aux_atom[i] < 0 || p->aux_atom[i] >= p->n_atoms) return fail(GW_ERR_ARG, "aux_atom out of range");
    if (i && p->aux_atom[i] < p->aux_atom[i - 1]) return fail(GW_ERR_ARG, "aux_atom must be non-decreasing");
  }
  return GW_OK;
}

// A batch plan routes a per-system call to the plan of system `sys`: the call starts after the
// work queued on the caller's stream and returns after its own work on the system's stream.
struct Route {
  gw_plan_s* P = nullptr;
  ~Route() {
    if (P) cudaStreamSynchronize(P->st);
  }
};

bool route(gw_plan& P, int32_t& sys, Route& r, gw_status* s) {
  if (P && !P->subs.empty()) {
    if (sys < 0 || sys >= (int)P->subs.size()) {
      *s = fail(GW_ERR_ARG, "sys out of range");
      return false;
    }
    cudaStreamSynchronize(P->st);
    P = P->subs[sys];
    sys = 0;
    r.P = P;
  }
  return true;
}

bool plan_ok(gw_plan P, int32_t sys, gw_status* s) {
  if (!P) {
    *s = fail(GW_ERR_ARG, "plan is NULL");
    return false;
  }
  if (P->err) {
    *s = fail(GW_ERR_STATE, "plan is in an error state from an earlier call");
    return false;
  }
  if (sys != 0) {
    *s = fail(GW_ERR_ARG, "sys out of range");
    return false;
  }
  return true;
}

}  // namespace

extern "C" {

const char* gw_last_error(void) { return g_last_error.c_str(); }

size_t gw_problem_bytes(void) { return sizeof(gw_problem); }

gw_status gw_device_allocations(uint64_t* count) {
  if (!count) return fail(GW_ERR_ARG, "count is NULL");
  *count = g_alloc_count.load();
  return GW_OK;
}

gw_status gw_kernel_launches(uint64_t* count) {
  if (!count) return fail(GW_ERR_ARG, "count is NULL");
  *count = (uint64_t)::gw::g_launch_count;
  return GW_OK;
}

gw_status gw_plan_create(const gw_problem* prob, int32_t n_sys, void* stream, gw_plan* out) {
  if (!out) return fail(GW_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n_sys < 1 || n_sys > 4096) return fail(GW_ERR_ARG, "n_sys out of range [1, 4096]");
  if (n_sys > 1) {
    if (!prob) return fail(GW_ERR_ARG, "problem array is NULL");
    gw_plan_s* B = new (std::nothrow) gw_plan_s();
    if (!B) return fail(GW_ERR_NOMEM, "host allocation failed");
    B->st = static_cast<cudaStream_t>(stream);
    GW_CUDA(cudaStreamSynchronize(B->st));   // inputs the caller queued on its stream
    for (int i = 0; i < n_sys; ++i) {
      cudaStream_t si = nullptr;
      gw_plan_s* sub = nullptr;
      gw_status st = GW_OK;
      if (cudaStreamCreateWithFlags(&si, cudaStreamNonBlocking) != cudaSuccess) {
        st = fail(GW_ERR_CUDA, "stream creation failed");
      } else {
        B->sub_streams.push_back(si);
        st = gw_plan_create(prob + i, 1, si, &sub);
      }
      if (st != GW_OK) {
        const std::string msg = "system " + std::to_string(i) + ": " + g_last_error;
        gw_plan_destroy(B);
        return fail(st, msg);
      }
      sub->group_budget = 2.0e9;
      B->subs.push_back(sub);
    }
    *out = B;
    return GW_OK;
  }
  GW_TRY(validate(prob, n_sys));
  gw_plan_s* P = new (std::nothrow) gw_plan_s();
  if (!P) return fail(GW_ERR_NOMEM, "host allocation failed");
  P->p = *prob;
  P->prec = prob->prec;
  P->fp64 = prob->prec == GW_FP64;
  P->st = static_cast<cudaStream_t>(stream);
  P->NK = prob->nk[0] * prob->nk[1] * prob->nk[2];
  P->N = prob->n_aux;
  P->NB = prob->n_basis;
  P->NBd = prob->n_bands;
  P->nocc = prob->n_occ;
  P->nunocc = prob->n_bands - prob->n_occ;
  P->nsig = prob->sigma_hi - prob->sigma_lo;
  P->nw = prob->n_freq;
  P->natoms = prob->n_atoms;
  P->basis_atom.assign(prob->basis_atom, prob->basis_atom + prob->n_basis);
  P->aux_atom.assign(prob->aux_atom, prob->aux_atom + prob->n_aux);
  P->R.assign(prob->R, prob->R + 3 * prob->n_R);
  P->p.basis_atom = P->basis_atom.data();
  P->p.aux_atom = P->aux_atom.data();
  P->p.R = P->R.data();
  P->p.freq = nullptr;   // the grid itself lives in P->freq / P->fweight
  P->p.freq_w = nullptr;
  if (const char* v = std::getenv("GW_WORKSPACE_LIMIT")) {
    const double lim = std::atof(v);
    if (lim > 0) P->ws_limit = (size_t)lim;
  }
  auto cleanup = [&](gw_status s) {
    std::string msg = g_last_error;
    gw_plan_destroy(P);
    g_last_error = msg;
    return s;
  };
  if (cudaGetDevice(&P->dev) != cudaSuccess) return cleanup(fail(GW_ERR_CUDA, "cudaGetDevice failed"));
  // geometry
  LriGeom& g = P->geom;
  g.n_atoms = P->natoms;
  g.NK = P->NK;
  g.NB = P->NB;
  g.NBd = P->NBd;
  g.N = P->N;
  g.nR = prob->n_R;
  for (int d = 0; d < 3; ++d) {
    g.nk[d] = prob->nk[d];
    g.koff[d] = prob->k_offset[d];
  }
  long long coff = 0, toff = 0;
  for (int A = 0; A < P->natoms; ++A) {
    int b0 = -1, nb = 0, x0 = -1, nx = 0;
    for (int i = 0; i < P->NB; ++i)
      if (P->basis_atom[i] == A) {
        if (b0 < 0) b0 = i;
        ++nb;
      }
    for (int i = 0; i < P->N; ++i)
      if (P->aux_atom[i] == A) {
        if (x0 < 0) x0 = i;
        ++nx;
      }
    if (nb == 0 || nx == 0) return cleanup(fail(GW_ERR_ARG, "every atom needs >= 1 basis and >= 1 aux function"));
    g.atom_b0[A] = b0;
    g.atom_nb[A] = nb;
    g.atom_x0[A] = x0;
    g.atom_nx[A] = nx;
    g.ctil_off[A] = coff;
    g.t_off[A] = toff;
    coff += (long long)prob->n_R * nx * nb * P->NB;
    toff += (long long)P->NK * nx * nb * P->NBd;
  }
  for (int r = 0; r < prob->n_R; ++r)
    for (int d = 0; d < 3; ++d) g.R[r][d] = P->R[3 * r + d];
  // frequency grid: the caller's, or the modified Gauss-Legendre grid of scale omega0
  P->freq.resize(P->nw);
  P->fweight.resize(P->nw);
  if (prob->freq) {
    for (int j = 0; j < P->nw; ++j) {
      P->freq[j] = prob->freq[j];
      P->fweight[j] = prob->freq_w[j];
    }
  } else {
    std::vector<double> x, w;
    gauss_legendre(P->nw, x, w);
    for (int j = 0; j < P->nw; ++j) {
      P->freq[j] = prob->omega0 * (1.0 + x[j]) / (1.0 - x[j]);
      P->fweight[j] = 2.0 * prob->omega0 * w[j] / ((1.0 - x[j]) * (1.0 - x[j]));
    }
  }
  const int N = P->N, nw = P->nw;
  const size_t NN = (size_t)N * N;
  gw_status s;
#define ALLOC(ptr, n)                                 \
  do {                                                \
    s = dalloc(P, &ptr, (n));                         \
    if (s != GW_OK) return cleanup(s);                \
  } while (0)
  ALLOC(P->d_freq, nw);
  ALLOC(P->d_fw, nw);
  ALLOC(P->d_mu, 1);
  ALLOC(P->d_status, 1);
  ALLOC(P->d_Vh, NN * P->NK);
  ALLOC(P->d_chi0, NN * nw);
  ALLOC(P->d_E, NN * nw);
  ALLOC(P->d_Wc, NN * nw);
  ALLOC(P->d_work, NN * nw);
  ALLOC(P->d_tmp, NN * nw);
  ALLOC(P->d_sigma, (size_t)P->NK * P->nsig * nw);
  ALLOC(P->d_head, nw);
  ALLOC(P->d_h, (size_t)nw * N);
  if (P->fp64) {
    c128* t;
    ALLOC(t, (size_t)toff);
    P->d_T1 = t;
  } else {
    c64* t;
    ALLOC(t, (size_t)toff);
    P->d_T1 = t;
  }
  if (prob->head_wings) {
    ALLOC(P->d_Vb0, NN);
    ALLOC(P->d_x1, N);
    ALLOC(P->d_v1, 1);
  }
  // chunk sizes: ~512 MB per M-type buffer
  const size_t esz = P->fp64 ? sizeof(c128) : sizeof(c64);
  const size_t budget = 512ull << 20;
  const long long rows_chi = (long long)P->nocc * P->nunocc;
  P->chi_nkk = (int)std::max<long long>(1, std::min<long long>(P->NK, budget / (rows_chi * N * esz)));
  P->ldm = ((rows_chi * P->chi_nkk + 31) / 32) * 32;
  const long long rows_sig = (long long)P->nsig * P->NBd;
  P->sig_nkk = (int)std::max<long long>(1, std::min<long long>(P->NK, budget / (rows_sig * N * esz)));
  P->sig_rows = rows_sig * P->sig_nkk;
  if (P->fp64) {
    c128 *a, *b, *c;
    ALLOC(a, (size_t)N * P->ldm);
    ALLOC(b, (size_t)P->sig_rows * N);
    ALLOC(c, (size_t)P->sig_rows * N);
    P->d_M = a;
    P->d_A = b;
    P->d_U = c;
    ALLOC(P->d_S_d, (size_t)P->sig_rows * nw);
  } else {
    c64 *a, *b;
    P->Kx = ((N + 31) / 32) * 32;
    ALLOC(a, (size_t)N * P->ldm);
    ALLOC(b, (size_t)P->sig_rows * P->Kx);   // raw plane of the Sigma rows, zero beyond n_aux
    P->d_M = a;
    P->d_A = b;
    ALLOC(P->d_S_f, (size_t)P->sig_rows * nw);
    for (int i = 0; i < 2; ++i) {
      uint8_t* pp;
      ALLOC(pp, (size_t)P->sig_rows * 2 * P->Kx * (P->prec == GW_3XTF32 ? 4 : 2));
      P->d_Apl[i] = pp;
    }
    const size_t we = (size_t)nw * N * 2 * P->Kx * (P->prec == GW_3XTF32 ? 4 : 2);
    for (int i = 0; i < (P->prec == GW_3XTF32 ? 4 : 6); ++i) {
      uint8_t* pp;
      ALLOC(pp, we);
      P->d_Wpl.b[i] = pp;
    }
    c64 *v32, *b32;
    ALLOC(v32, NN * P->NK);
    P->d_Vh32 = v32;
    if (prob->head_wings) {
      ALLOC(b32, NN);
      P->d_Vb32 = b32;
    }
  }
  if (!P->fp64) {
    const size_t pe = (size_t)N * 2 * P->ldm * (P->prec == GW_3XTF32 ? 4 : 2);
    ALLOC(P->d_Praw, (size_t)N * 2 * P->ldm);
    P->n_bpl = P->prec == GW_3XBF16 ? 3 : 2;
    ALLOC(P->d_absmax, 1);
    {
      const size_t kp = (size_t)(N + 31) / 32 * 32;
      ALLOC(P->d_hb[0], (size_t)nw * N * 2 * kp);
      ALLOC(P->d_hb[1], (size_t)nw * N * 2 * kp);
      ALLOC(P->d_hones, kp);
      ALLOC(P->d_hesc, (size_t)nw);
    }
    ALLOC(P->d_eB, 1);
    ALLOC(P->d_escale, (size_t)nw);
    for (int i = 0; i < P->n_bpl; ++i) {
      uint8_t* pp;
      ALLOC(pp, pe);
      P->d_Pb[i] = pp;
    }
    ALLOC(P->d_wtab, (size_t)nw * P->ldm);
    if (const char* e = std::getenv("GW_CHI0_SEG_ROWS")) P->seg_rows = std::max(32, std::atoi(e));
    if (const char* e = std::getenv("GW_CHI0_COMPRESS_TOL")) P->compress_tol = std::max(0.0, std::atof(e));
    if (nw <= 64) {
      ALLOC(P->d_wG, (size_t)nw * nw * P->NK);
      ALLOC(P->d_wU, (size_t)nw * nw * P->NK);
      ALLOC(P->d_wlam, (size_t)nw * P->NK);
      ALLOC(P->d_wn, (size_t)nw * P->NK);
      ALLOC(P->d_wE, (size_t)nw * nw * P->NK);
      ALLOC(P->d_wP, (size_t)nw * nw * P->NK);
      ALLOC(P->d_werr, (size_t)nw * (nw + 1) * P->NK);
      ALLOC(P->d_C, (size_t)nw * NN);
    }
  }
  ALLOC(P->d_delta, P->ldm);
  ALLOC(P->d_delta_f, P->ldm);
  ALLOC(P->d_pq, P->ldm);
  if (prob->head_wings == 2) {
    ALLOC(P->d_pq3, 3 * (size_t)P->ldm);
    ALLOC(P->d_A6, (size_t)nw * 6);
    ALLOC(P->d_h3, (size_t)nw * 3 * N);
    ALLOC(P->d_Y3, (size_t)nw * 3 * N);
    ALLOC(P->d_G3, (size_t)nw * 3 * N);
    ALLOC(P->d_m10, (size_t)nw * 10);
    // direction rule: 8 Gauss-Legendre nodes in cos(theta) x 16 equally spaced phi (half-step
    // offset), weights summing to one; symmetric under q^ -> -q^
    std::vector<double> u, wu, rule;
    gauss_legendre(8, u, wu);
    for (int i = 0; i < 8; ++i)
      for (int j = 0; j < 16; ++j) {
        const double ph = 2.0 * M_PI * (j + 0.5) / 16.0, st = std::sqrt(1.0 - u[i] * u[i]);
        rule.insert(rule.end(), {st * std::cos(ph), st * std::sin(ph), u[i], wu[i] / 2.0 / 16.0});
      }
    P->n_dirs = 128;
    ALLOC(P->d_dirs, rule.size());
    if (cudaMemcpy(P->d_dirs, rule.data(), sizeof(double) * rule.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return cleanup(fail(GW_ERR_CUDA, "direction rule upload failed"));
  }
#undef ALLOC
  if (cudaEventCreate(&P->ev0) != cudaSuccess || cudaEventCreate(&P->ev1) != cudaSuccess)
    return cleanup(fail(GW_ERR_CUDA, "cudaEventCreate failed"));
  cudaStream_t st = P->st;
#define CK(call)                                                                                     \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) return cleanup(fail(GW_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_))); \
  } while (0)
  CK(cudaMemcpyAsync(P->d_freq, P->freq.data(), nw * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(P->d_fw, P->fweight.data(), nw * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(P->d_status, 0, sizeof(int), st));
  CK(cudaMemsetAsync(P->d_sigma, 0, sizeof(c128) * (size_t)P->NK * P->nsig * nw, st));
  // chemical potential
  if (std::isnan(prob->mu)) {
    launch_midgap(P->NK, P->NBd, P->nocc, prob->eps, P->d_mu, st);
  } else {
    CK(cudaMemcpyAsync(P->d_mu, &prob->mu, sizeof(double), cudaMemcpyHostToDevice, st));
  }
  CK(cudaMemcpyAsync(&P->mu, P->d_mu, sizeof(double), cudaMemcpyDeviceToHost, st));
  // half-transformed LRI coefficients
  if (P->fp64)
    launch_lri_halfT<double>(g, prob->ctil_R, reinterpret_cast<const c128*>(prob->evec),
                             static_cast<c128*>(P->d_T1), nullptr, st);
  else
    launch_lri_halfT<float>(g, prob->ctil_R, reinterpret_cast<const c128*>(prob->evec), static_cast<c64*>(P->d_T1),
                            nullptr, st);
  if ((s = check_launch(P, "lri_halfT")) != GW_OK) return cleanup(s);
  // time-reversal symmetry of the inputs, when the caller declares it
  if (prob->time_reversal) {
    unsigned long long* d_chk = nullptr;
    if ((s = dalloc(P, &d_chk, 4)) != GW_OK) return cleanup(s);
    CK(cudaMemsetAsync(d_chk, 0, 4 * sizeof(unsigned long long), st));
    ++g_launch_count, k_trs_check<<<152 * 8, 256, 0, st>>>(prob->nk[0], prob->nk[1], prob->nk[2], P->NBd, prob->eps, N,
                                                            reinterpret_cast<const c128*>(prob->V), d_chk);
    unsigned long long h[4] = {0, 0, 0, 0};
    CK(cudaMemcpyAsync(h, d_chk, sizeof(h), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double v[4];
    for (int i = 0; i < 4; ++i) std::memcpy(&v[i], &h[i], sizeof(double));
    if (!(v[0] <= 1e-12 * std::max(v[1], 1.0)) || !(v[2] <= 1e-12 * std::max(v[3], 1e-300)))
      return cleanup(fail(GW_ERR_ARG, "time_reversal is set but eps(-k) != eps(k) or V(-q) != conj(V(q)) (max "
                                      "differences " + std::to_string(v[0]) + ", " + std::to_string(v[2]) + ")"));
    P->trs = true;
    if (prob->head_wings != 1) {
      std::vector<int> rep, isrep(P->NK, 0);
      for (int k = 0; k < P->NK; ++k) {
        const int i3 = k % prob->nk[2], i2 = (k / prob->nk[2]) % prob->nk[1], i1 = k / (prob->nk[1] * prob->nk[2]);
        const int mk = (((prob->nk[0] - i1) % prob->nk[0]) * prob->nk[1] + (prob->nk[1] - i2) % prob->nk[1]) *
                           prob->nk[2] + (prob->nk[2] - i3) % prob->nk[2];
        if (mk >= k) {
          rep.push_back(k);
          isrep[k] = 1;
        }
      }
      P->n_krep = (int)rep.size();
      if ((s = dalloc(P, &P->d_ktab, rep.size())) != GW_OK) return cleanup(s);
      if ((s = dalloc(P, &P->d_isrep, isrep.size())) != GW_OK) return cleanup(s);
      if ((s = dalloc(P, &P->d_sigtmp, (size_t)P->NK * P->nsig * nw)) != GW_OK) return cleanup(s);
      CK(cudaMemcpy(P->d_ktab, rep.data(), sizeof(int) * rep.size(), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(P->d_isrep, isrep.data(), sizeof(int) * isrep.size(), cudaMemcpyHostToDevice));
    }
  }
  // V(q)^1/2; at q = 0 with head_wings split off the lambda = 1 eigenvector first
  const c128* V = reinterpret_cast<const c128*>(prob->V);
  CK(cudaMemcpyAsync(P->d_Vh, V, sizeof(c128) * NN * P->NK, cudaMemcpyDeviceToDevice, st));
  double t_shift = 1.0;
  if (prob->head_wings) {
    launch_power_iter(N, V, P->d_x1, P->d_v1, 200, st);
    CK(cudaMemcpyAsync(&P->h_v1, P->d_v1, sizeof(double), cudaMemcpyDeviceToHost, st));
    std::vector<c128> diag(N);
    CK(cudaMemcpy2DAsync(diag.data(), sizeof(c128), V, sizeof(c128) * (N + 1), sizeof(c128), N,
                         cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double tr = 0;
    for (int i = 0; i < N; ++i) tr += diag[i].re;
    t_shift = N > 1 ? std::max(1e-3, (tr - P->h_v1) / (N - 1)) : 1.0;
    // B = V(0) - v1 x1 x1^H + t x1 x1^H
    launch_rank1(N, P->d_Vh, P->d_x1, t_shift - P->h_v1, st);
  }
  if (P->fp64)
    s = newton_schulz<double>(P, P->d_Vh, P->d_Vh, P->NK, 24);
  else if (N % 2 == 0)
    s = newton_schulz_tc(P, P->d_Vh, P->NK, 24);
  else
    s = newton_schulz<float>(P, P->d_Vh, P->d_Vh, P->NK, 24);
  if (s != GW_OK) return cleanup(s);
  if (prob->head_wings) {
    // Vb0 = sqrt(B) - sqrt(t) x1 x1^H ;  Vh(0) = Vb0 + sqrt(v1) x1 x1^H
    launch_rank1(N, P->d_Vh, P->d_x1, -std::sqrt(t_shift), st);
    CK(cudaMemcpyAsync(P->d_Vb0, P->d_Vh, sizeof(c128) * NN, cudaMemcpyDeviceToDevice, st));
    launch_rank1(N, P->d_Vh, P->d_x1, std::sqrt(std::max(P->h_v1, 0.0)), st);
  }
  if (!P->fp64) {
    launch_convert((int)(NN * P->NK), P->d_Vh, P->d_Vh32, st);
    if (prob->head_wings) launch_convert((int)NN, P->d_Vb0, P->d_Vb32, st);
    CK(cudaMemsetAsync(P->d_A, 0, sizeof(c64) * (size_t)P->sig_rows * P->Kx, st));
  }
  if ((s = check_launch(P, "plan setup")) != GW_OK) return cleanup(s);
  CK(cudaStreamSynchronize(st));
#undef CK
  *out = P;
  return GW_OK;
}

gw_status gw_plan_destroy(gw_plan P) {
  if (!P) return GW_OK;
  if (!P->subs.empty() || !P->sub_streams.empty()) {
    for (gw_plan_s* sub : P->subs) gw_plan_destroy(sub);
    for (cudaStream_t si : P->sub_streams) cudaStreamDestroy(si);
    delete P;
    return GW_OK;
  }
  if (P->st) cudaStreamSynchronize(P->st);
  else cudaDeviceSynchronize();
  for (void* a : P->allocs) cudaFree(a);
  if (P->chi0plan) chi0_plan_free(P->chi0plan);
  if (P->ev0) cudaEventDestroy(P->ev0);
  if (P->ev1) cudaEventDestroy(P->ev1);
  for (auto& e : P->evs) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  delete P;
  return GW_OK;
}

gw_status gw_plan_freq(gw_plan P, double* freq, double* weight) {
  if (P && !P->subs.empty()) P = P->subs[0];  // batch plan: system 0
  if (!P) return fail(GW_ERR_ARG, "plan is NULL");
  if (freq) std::copy(P->freq.begin(), P->freq.end(), freq);
  if (weight) std::copy(P->fweight.begin(), P->fweight.end(), weight);
  return GW_OK;
}

gw_status gw_plan_mu(gw_plan P, double* mu) {
  if (P && !P->subs.empty()) P = P->subs[0];  // batch plan: system 0
  if (!P || !mu) return fail(GW_ERR_ARG, "NULL argument");
  *mu = P->mu;
  return GW_OK;
}

gw_status gw_plan_chi0_terms(gw_plan P, int32_t* terms) {
  if (P && !P->subs.empty()) P = P->subs[0];  // batch plan: system 0
  if (!P || !terms) return fail(GW_ERR_ARG, "NULL argument");
  *terms = P->last_T;
  return GW_OK;
}

gw_status gw_plan_last_chi0_stats(gw_plan P, double* ms, double* flops) {
  if (P && !P->subs.empty()) P = P->subs[0];  // batch plan: system 0
  if (!P) return fail(GW_ERR_ARG, "plan is NULL");
  if (ms) *ms = P->last_chi0_ms;
  if (flops) *flops = P->last_chi0_flops;
  return GW_OK;
}

}  // extern "C"

namespace {

// chi0(q) into `chi0` ([nw][N][N], FP64). Records CUDA events around the contraction launches.
bool compress_on(const gw_plan_s* P) {
  return !P->fp64 && P->compress_tol > 0.0 && P->d_wG && P->nw >= 4 && P->nw <= 64;
}

// Weight bases of q0 .. q0+nq-1 for the frequency compression of chi0: the Gram matrix of the
// weight rows over all pair rows of q (FP64), normalised, its eigen-decomposition (one batched
// Jacobi), the expansion / projection matrices, and T_q = the smallest number of components whose
// per-frequency residual (computed directly over all pair rows) is within compress_tol for every
// frequency. One host synchronisation per call.
gw_status chi0_prepare(gw_plan_s* P, const int* qs, int nq) {
  if (!compress_on(P)) return GW_OK;
  cudaStream_t st = P->st;
  const int nw = P->nw, na = P->nunocc, nb = P->nocc;
  const long long sG = (long long)nw * nw;
  GW_CUDA(cudaMemsetAsync(P->d_wG, 0, sizeof(c128) * sG * nq, st));
  for (int j = 0; j < nq; ++j) {
    for (int kk0 = 0; kk0 < P->NK; kk0 += P->chi_nkk) {
      const int nkk = std::min(P->chi_nkk, P->NK - kk0);
      launch_pairs(P->NK, P->NBd, P->p.nk, qs[j], kk0, nkk, P->nocc, na, 0, nb, P->p.eps, nullptr, P->p.qhat,
                   P->d_delta, P->d_delta_f, nullptr, st);
      launch_wgram(nkk * na * nb, nw, P->d_delta, P->d_freq, P->d_wG + j * sG, st);
    }
  }
  launch_wnorm(nw, nq, P->d_wG, P->d_wn, st);
  launch_small_jacobi(nw, nq, P->d_wG, P->d_wlam, P->d_wU, st);
  launch_wproj(nw, nq, P->d_wU, P->d_wn, P->d_wE, P->d_wP, st);
  const long long sE = (long long)nw * (nw + 1);
  GW_CUDA(cudaMemsetAsync(P->d_werr, 0, sizeof(double) * sE * nq, st));
  for (int j = 0; j < nq; ++j) {
    for (int kk0 = 0; kk0 < P->NK; kk0 += P->chi_nkk) {
      const int nkk = std::min(P->chi_nkk, P->NK - kk0);
      launch_pairs(P->NK, P->NBd, P->p.nk, qs[j], kk0, nkk, P->nocc, na, 0, nb, P->p.eps, nullptr, P->p.qhat,
                   P->d_delta, P->d_delta_f, nullptr, st);
      launch_wresid(nkk * na * nb, nw, P->d_delta, P->d_freq, P->d_wE + j * sG, P->d_wP + j * sG, P->d_werr + j * sE,
                    st);
    }
  }
  std::vector<double> er((size_t)sE * nq);
  GW_CUDA(cudaMemcpyAsync(er.data(), P->d_werr, sizeof(double) * er.size(), cudaMemcpyDeviceToHost, st));
  GW_CUDA(cudaStreamSynchronize(st));
  P->comp_T.assign(nq, nw);
  for (int j = 0; j < nq; ++j) {
    const double* e = er.data() + (size_t)j * sE;
    for (int T = 1; T <= nw; ++T) {
      double worst = 0.0;
      for (int f = 0; f < nw; ++f) {
        const double n2 = e[f * (nw + 1)];
        if (n2 > 0.0) worst = std::max(worst, std::sqrt(std::max(e[f * (nw + 1) + T], 0.0) / n2));
      }
      if (worst <= P->compress_tol) {
        P->comp_T[j] = T;
        break;
      }
    }
  }
  P->comp_qs.assign(qs, qs + nq);
  P->comp_nw = nw;
  return check_launch(P, "chi0 weight spectra");
}

gw_status chi0_core(gw_plan_s* P, int q, c128* chi0) {
  cudaStream_t st = P->st;
  const int N = P->N, nw = P->nw;
  const size_t NN = (size_t)N * N;
  const c128* evec = reinterpret_cast<const c128*>(P->p.evec);
  GW_CUDA(cudaMemsetAsync(chi0, 0, sizeof(c128) * NN * nw, st));
  const bool hw = P->p.head_wings && q == 0;
  const bool hw_avg = hw && P->p.head_wings == 2;
  if (hw) {
    std::vector<double> ones(nw, 1.0);
    GW_CUDA(cudaMemcpyAsync(P->d_head, ones.data(), nw * sizeof(double), cudaMemcpyHostToDevice, st));
    GW_CUDA(cudaStreamSynchronize(st));
    GW_CUDA(cudaMemsetAsync(P->d_h, 0, sizeof(c128) * nw * N, st));
  }
  if (hw_avg) {
    GW_CUDA(cudaMemsetAsync(P->d_A6, 0, sizeof(double) * nw * 6, st));
    GW_CUDA(cudaMemsetAsync(P->d_h3, 0, sizeof(c128) * nw * 3 * N, st));
  }
  // Cartesian p . e_a tables of the chunk (direction-averaged q = 0)
  auto pairs3 = [&](int kk0, int nkk) {
    for (int a = 0; a < 3; ++a) {
      const double e[3] = {a == 0 ? 1.0 : 0.0, a == 1 ? 1.0 : 0.0, a == 2 ? 1.0 : 0.0};
      launch_pairs(P->NK, P->NBd, P->p.nk, q, kk0, nkk, P->nocc, P->nunocc, 0, P->nocc, P->p.eps,
                   reinterpret_cast<const c128*>(P->p.pmom), e, nullptr, nullptr, P->d_pq3 + a * P->ldm, st);
    }
  };
  const double hw_pref = 4.0 * M_PI * P->p.spin / (P->p.omega_cell * P->NK);
  const double scale = -P->p.spin / P->NK;
  const int na = P->nunocc, nb = P->nocc;
  // frequency compression (split precision): chi0(w_j) = sum_t U_jt C_t over T <= nw weight rows
  const bool comp = compress_on(P);
  int jq = 0;                 // position of q in the list of prepared weight bases
  int T = nw;
  const double* Uw = nullptr;
  if (comp) {
    jq = (int)(std::find(P->comp_qs.begin(), P->comp_qs.end(), q) - P->comp_qs.begin());
    if (jq == (int)P->comp_qs.size() || P->comp_nw != nw) {
      GW_TRY(chi0_prepare(P, &q, 1));
      jq = 0;
    }
    T = P->comp_T[jq];
    Uw = P->d_wE + (long long)jq * nw * nw;
    P->last_T = T;
    GW_CUDA(cudaMemsetAsync(P->d_C, 0, sizeof(c128) * NN * T, st));
  }
  for (int kk0 = 0; kk0 < P->NK; kk0 += P->chi_nkk) {
    const int nkk = std::min(P->chi_nkk, P->NK - kk0);
    const int K = nkk * na * nb;
    cudaEvent_t e0, e1;
    GW_TRY(P->event_pair(e0, e1));
    launch_pairs(P->NK, P->NBd, P->p.nk, q, kk0, nkk, P->nocc, na, 0, nb, P->p.eps,
                 reinterpret_cast<const c128*>(P->p.pmom), P->p.qhat, P->d_delta, P->d_delta_f,
                 hw ? P->d_pq : nullptr, st);
    if (P->fp64) {
      c128* M = static_cast<c128*>(P->d_M);
      launch_mgen<double>(P->geom, static_cast<const c128*>(P->d_T1), nullptr, evec, q, kk0, nkk, MAP_K_IS_KK,
                          P->nocc, na, 0, nb, M, 1, P->ldm, st);
      GW_CUDA(cudaEventRecord(e0, st));
      launch_chi0_simt<double>(N, K, M, P->ldm, nullptr, P->d_delta, P->d_freq, nw, scale, chi0, st);
      GW_CUDA(cudaEventRecord(e1, st));
      // one direction (head_wings = 1) or the three Cartesian components for the average
      if (hw && !hw_avg)
        launch_head_wings<double>(N, K, M, P->ldm, P->d_delta, P->d_pq, P->d_freq, nw, hw_pref, P->d_head, P->d_h,
                                  st);
      if (hw_avg) {
        pairs3(kk0, nkk);
        launch_head_wings3<double>(N, K, M, P->ldm, P->d_delta, P->d_pq3, P->ldm, P->d_freq, nw, hw_pref, P->d_A6,
                                   P->d_h3, st);
      }
    } else {
      // the fp32 plane of M [N][2*ldm] (zero rows beyond K), its split pieces, then the tcgen05
      // contraction
      const int kind = P->prec == GW_3XFP16 ? 0 : (P->prec == GW_3XBF16 ? 1 : 2);
      if (K < P->ldm) {
        // zero the padding pair rows K .. ldm-1 of the plane (and their transition energies)
        const size_t pad = (size_t)(P->ldm - K) * 2;
        GW_CUDA(cudaMemset2DAsync(P->d_Praw + 2 * (size_t)K, 2 * P->ldm * sizeof(float), 0, pad * sizeof(float), N,
                                  st));
        GW_CUDA(cudaMemsetAsync(P->d_delta_f + K, 0, sizeof(float) * (P->ldm - K), st));
      }
      GW_CUDA(cudaMemsetAsync(P->d_absmax, 0, sizeof(unsigned), st));
      if (!launch_mgen_chi(P->geom, static_cast<const c64*>(P->d_T1), evec, q, kk0, nkk, P->nocc, na, 0, nb,
                           P->d_Praw, 2 * P->ldm, 0, P->d_absmax, st) &&
          !P->mtune.run(1, na, nb, st, [&](int v) {
            launch_mgen_planes(P->geom, static_cast<const c64*>(P->d_T1), evec, q, kk0, nkk, P->nocc, na, 0, nb,
                               P->d_Praw, nullptr, 2 * P->ldm, 0, 0, st, v, P->d_absmax);
          }))
        return fail(GW_ERR_CUDA, "M kernel autotuner: CUDA error");
      Chi0hArgs a{};
      a.kind = kind;
      a.N = N;
      a.Kpad = (int)P->ldm;
      a.T = comp ? T : nw;
      a.raw = P->d_Praw;
      for (int i = 0; i < P->n_bpl; ++i) a.bpl[i] = P->d_Pb[i];
      a.absmax = P->d_absmax;
      a.eB = P->d_eB;
      a.wtab = P->d_wtab;
      a.escale = P->d_escale;
      a.scale = scale;
      a.out = comp ? P->d_C : chi0;
      a.status = P->d_status;
      a.seg_rows = P->seg_rows;
      cudaEvent_t ev[2] = {e0, e1};
      a.events = ev;
      GW_TRY(chi0h_pieces(a, st) == GW_OK ? GW_OK : fail(GW_ERR_CUDA, "chi0 operand pieces: launch failed"));
      if (comp)
        launch_wtab_compressed(K, (int)P->ldm, nw, T, P->d_delta, P->d_freq,
                               P->d_wP + (long long)jq * nw * nw, P->d_wtab, st);
      else
        chi0h_weights(K, (int)P->ldm, nw, P->d_delta_f, P->d_freq, P->d_wtab, st);
      std::string err;
      gw_status ts = chi0h_run(a, &P->chi0plan, st, err);
      if (ts != GW_OK) {
        P->err = 1;
        return fail(ts, err);
      }
      if (hw) {
        c64* M = static_cast<c64*>(P->d_M);
        if (!P->mtune.run(0, na, nb, st, [&](int v) {
              launch_mgen<float>(P->geom, static_cast<const c64*>(P->d_T1), nullptr, evec, q, kk0, nkk, MAP_K_IS_KK,
                                 P->nocc, na, 0, nb, M, 1, P->ldm, st, v);
            }))
          return fail(GW_ERR_CUDA, "M kernel autotuner: CUDA error");
        if (!hw_avg)
          launch_head_wings<float>(N, K, M, P->ldm, P->d_delta, P->d_pq, P->d_freq, nw, hw_pref, P->d_head, P->d_h,
                                   st);
        else {
          pairs3(kk0, nkk);
          launch_head_wings3<float>(N, K, M, P->ldm, P->d_delta, P->d_pq3, P->ldm, P->d_freq, nw, hw_pref, P->d_A6,
                                    P->d_h3, st);
        }
      }
    }
    GW_TRY(check_launch(P, "chi0"));
  }
  if (comp) launch_expand(nw, T, (long long)NN, Uw, P->d_C, chi0, st);
  if (!P->fp64) tc_herm_fill(N, nw, chi0, st);
  P->chi0_flops_acc += 8.0 * (double)P->NK * na * nb * ((double)N * (N + 1) / 2) * nw;
  return GW_OK;
}

// C[b] = alpha A[b] H[b] for b < nb on the tensor cores (split precision screen products; H
// Hermitian, FP64 or FP32)
gw_status herm_gemm(gw_plan_s* P, const c64* A, bool a_batch, const c128* H64, const c64* H32, bool h_batch,
                    double alpha, c128* C, int nb) {
  HermGemmArgs g{};
  g.N = P->N;
  g.nb = nb;
  g.A = A;
  g.a_batch = a_batch ? 1 : 0;
  g.H64 = H64;
  g.H32 = H32;
  g.h_batch = h_batch ? 1 : 0;
  g.alpha = alpha;
  g.C = C;
  g.bpl[0] = P->d_hb[0];
  g.bpl[1] = P->d_hb[1];
  g.ones = P->d_hones;
  g.escale = P->d_hesc;
  g.status = P->d_status;
  std::string err;
  gw_status ts = herm_gemm_run(g, &P->chi0plan, P->st, err);
  if (ts != GW_OK) {
    P->err = 1;
    return fail(ts, "screen product: " + err);
  }
  return GW_OK;
}
gw_status herm_gemm(gw_plan_s* P, const c64* A, bool a_batch, const c128* H, bool h_batch, double alpha, c128* C) {
  return herm_gemm(P, A, a_batch, H, nullptr, h_batch, alpha, C, P->nw);
}

// eps~(q) = 1 - V^1/2 chi0 V^1/2 (head and wings at q = 0) into E ([nw][N][N], FP64)
gw_status eps_core(gw_plan_s* P, int q, const c128* chi0, c128* E) {
  cudaStream_t st = P->st;
  const int N = P->N, nw = P->nw;
  const long long NN = (long long)N * N;
  const bool hw = P->p.head_wings && q == 0;
  const c128* Vh = P->d_Vh + (long long)q * NN;
  const c128* Vin = hw ? P->d_Vb0 : Vh;     // V^1/2 entering eps~ (body only at q = 0)
  const c128 one{1, 0}, zero{0, 0}, mone{-1, 0};
  c64* A32 = reinterpret_cast<c64*>(P->d_work);
  if (P->fp64) {
    launch_zgemm<double>(N, N, N, one, chi0, N, NN, OP_N, Vin, N, 0, OP_N, zero, P->d_tmp, N, NN, nw, st);
    launch_zgemm<double>(N, N, N, mone, Vin, N, 0, OP_N, P->d_tmp, N, NN, OP_N, zero, E, N, NN, nw, st);
  } else {
    // V^1/2 chi0 V^1/2 as (V^1/2 chi0) V^1/2: both right operands are Hermitian, the form of the
    // tensor-core kernel (TF32 two-piece products, FP64 accumulation)
    const c64* Vh32 = P->d_Vh32 + (long long)q * NN;
    const c64* Vin32 = hw ? P->d_Vb32 : Vh32;
    GW_TRY(herm_gemm(P, Vin32, false, chi0, true, 1.0, P->d_tmp));
    launch_convert((int)(NN * nw), P->d_tmp, A32, st);
    GW_TRY(herm_gemm(P, A32, true, Vin, false, -1.0, E));
  }
  launch_axpby_identity<double>(N, E, NN, nw, 1.0, st);
  if (hw && P->p.head_wings == 1) {
    // Vbh[w] = Vb0 h[w], then the rank-2 head / wing correction
    launch_zgemm<double>(nw, N, N, one, P->d_h, N, 0, OP_N, P->d_Vb0, N, 0, OP_T, zero, P->d_tmp, N, 0, 1, st);
    const double c = (P->p.spin / P->NK) * std::sqrt(4.0 * M_PI / P->p.omega_cell);
    launch_q0_correction(N, nw, E, P->d_x1, P->d_tmp, P->d_head, c, st);
  }
  return check_launch(P, "eps~");
}

// Direction-averaged q = 0 (head_wings = 2; reading: the head and wings of Eq.
// dielectric_func_gamma depend on the direction of q -> 0, and eps~^-1 - 1 is averaged over the
// directions of a sphere rule). X holds G - 1 on entry, G the inverse of the body
// eps~_b = 1 - Vb0 chi0 Vb0 (x1 is its eigenvector with eigenvalue 1). For a direction q^ the wing
// column is y(q^) = sum_a q_a y_a, y_a = -c Vb0 h_a, and the head 1 + q^T A q^; the Schur complement
// s = 1 + q^T (A - Re Gamma) q^, Gamma_ab = y_a^H G y_b, gives
//   eps~(q^)^-1 - 1 = (G - 1) + (1/s - 1) x1 x1^H - (x1 g^H + g x1^H)/s + g g^H/s,  g = G y(q^),
// whose average over the rule needs only <1/s>, <q_a/s> and <q_a q_b/s> (k_q0avg_moments).
gw_status q0_average(gw_plan_s* P, c128* X) {
  cudaStream_t st = P->st;
  const int N = P->N, nw = P->nw;
  const long long NN = (long long)N * N;
  const double c = (P->p.spin / P->NK) * std::sqrt(4.0 * M_PI / P->p.omega_cell);
  launch_zgemm<double>(3 * nw, N, N, c128{-c, 0}, P->d_h3, N, 0, OP_N, P->d_Vb0, N, 0, OP_T, c128{0, 0}, P->d_Y3, N,
                       0, 1, st);
  launch_zgemm<double>(N, 3, N, c128{1, 0}, X, N, NN, OP_N, P->d_Y3, N, 3LL * N, OP_T, c128{0, 0}, P->d_G3, 3,
                       3LL * N, nw, st);
  launch_q0avg_moments(N, nw, P->d_Y3, P->d_G3, P->d_A6, P->d_dirs, P->n_dirs, P->d_m10, P->d_status, st);
  launch_q0avg_update(N, nw, X, NN, P->d_x1, P->d_G3, P->d_m10, st);
  return check_launch(P, "q = 0 direction average");
}

// W^c(q) = V^1/2 X V^1/2 with X = eps~^-1 - 1 ([nw][N][N], FP64 in and out)
gw_status w_core(gw_plan_s* P, int q, const c128* X, c128* Wc) {
  cudaStream_t st = P->st;
  const int N = P->N, nw = P->nw;
  const long long NN = (long long)N * N;
  const c128* Vh = P->d_Vh + (long long)q * NN;
  const c128 one{1, 0}, zero{0, 0};
  c64* A32 = reinterpret_cast<c64*>(P->d_work);
  if (P->fp64) {
    launch_zgemm<double>(N, N, N, one, X, N, NN, OP_N, Vh, N, 0, OP_N, zero, P->d_tmp, N, NN, nw, st);
    launch_zgemm<double>(N, N, N, one, Vh, N, 0, OP_N, P->d_tmp, N, NN, OP_N, zero, Wc, N, NN, nw, st);
  } else {
    // V^1/2 X V^1/2 as (V^1/2 X) V^1/2 (X = eps~^-1 - 1 and V^1/2 Hermitian)
    const c64* Vh32 = P->d_Vh32 + (long long)q * NN;
    GW_TRY(herm_gemm(P, Vh32, false, X, true, 1.0, P->d_tmp));
    launch_convert((int)(NN * nw), P->d_tmp, A32, st);
    GW_TRY(herm_gemm(P, A32, true, Vh, false, 1.0, Wc));
  }
  return check_launch(P, "W^c");
}

// q term of Sigma_c from W^c(q), accumulated into sig ([N_k][n_sigma][nw])
// target k in [k_lo, k_hi) (k_hi < 0: all)
// use_ktab: the target k of P->d_ktab (time reversal, Sigma_c(-k) = Sigma_c(k)) instead of a range
gw_status sigma_core(gw_plan_s* P, int q, const c128* Wc, c128* sig, bool conjW = false, int k_lo = 0, int k_hi = -1,
                     bool use_ktab = false) {
  cudaStream_t st = P->st;
  const int N = P->N, nw = P->nw, NBd = P->NBd, nsig = P->nsig;
  const long long NN = (long long)N * N;
  const c128* evec = reinterpret_cast<const c128*>(P->p.evec);
  const double pref = -1.0 / (2.0 * M_PI * P->NK);
  const int tf32 = P->prec == GW_3XTF32;
  if (!P->fp64) tc_w_planes(N, nw, P->Kx, Wc, P->d_Wpl, tf32, st, conjW ? 1 : 0);
  const int k_end = use_ktab ? P->n_krep : (k_hi < 0 ? P->NK : k_hi);
  LriGeom geom = P->geom;                 // the M kernels map row blocks to target k through ktab
  geom.ktab = use_ktab ? P->d_ktab : nullptr;
  const int* ktab = geom.ktab;
  for (int kk0 = use_ktab ? 0 : k_lo; kk0 < k_end; kk0 += P->sig_nkk) {
    const int nkk = std::min(P->sig_nkk, k_end - kk0);
    const int R = nkk * nsig * NBd;
    if (P->fp64) {
      c128* A = static_cast<c128*>(P->d_A);
      c128* U = static_cast<c128*>(P->d_U);
      launch_mgen<double>(geom, static_cast<const c128*>(P->d_T1), nullptr, evec, q, kk0, nkk,
                          MAP_K_IS_KK_MINUS_Q, P->p.sigma_lo, nsig, 0, NBd, A, N, 1, st);
      for (int j = 0; j < nw; ++j) {
        launch_zgemm<double>(R, N, N, c128{1, 0}, A, N, 0, OP_N, Wc + j * NN, N, 0, conjW ? OP_CONJ : OP_N,
                             c128{0, 0}, U, N, 0, 1, st);
        launch_rowdot<double>(R, N, U, A, N, nullptr, P->d_S_d, j, nw, st);
      }
    } else {
      // rows a_r as an fp32 plane [R][Kx] (zero beyond n_aux), then the tensor-core contraction
      c64* A = static_cast<c64*>(P->d_A);
      if (!launch_mgen_sig(geom, static_cast<const c64*>(P->d_T1), evec, q, kk0, nkk, P->p.sigma_lo, nsig, NBd, A,
                           P->Kx, 1, st) &&
          !P->mtune.run(0, nsig, NBd, st, [&](int v) {
            launch_mgen<float>(geom, static_cast<const c64*>(P->d_T1), nullptr, evec, q, kk0, nkk,
                               MAP_K_IS_KK_MINUS_Q, P->p.sigma_lo, nsig, 0, NBd, A, P->Kx, 1, st, v);
          }))
        return fail(GW_ERR_CUDA, "M kernel autotuner: CUDA error");
      GW_CUDA(cudaMemsetAsync(P->d_S_f, 0, sizeof(float) * (size_t)R * nw, st));
      TcSigmaArgs a{};
      a.R = R;
      a.N = N;
      a.Kpad = P->Kx;
      a.nw = nw;
      a.raw = reinterpret_cast<const float*>(A);
      for (int i = 0; i < 6; ++i) a.bpl[i] = P->d_Wpl.b[i];
      a.S = P->d_S_f;
      a.apl[0] = P->d_Apl[0];
      a.apl[1] = P->d_Apl[1];
      a.tf32 = tf32;
      a.status = P->d_status;
      std::string err;
      gw_status ts = tc_sigma_run(a, st, err);
      if (ts != GW_OK) {
        P->err = 1;
        return fail(ts, err);
      }
    }
    launch_sigma_conv_chunk(kk0, nkk, nsig, NBd, P->p.nk, q, P->p.eps, P->d_mu, P->d_S_f, P->d_S_d, P->d_freq,
                            P->d_fw, nw, pref, sig, P->fp64, st, ktab);
    GW_TRY(check_launch(P, "Sigma_c"));
  }
  return GW_OK;
}

gw_status g0w0_sur(gw_plan_s* P, c128* sig);  // the surrogate pass, defined below

// q-group buffers of gw_g0w0: chi0 (then W^c), eps~ (then eps~^-1 - 1), Cholesky scratch
gw_status ensure_groups(gw_plan_s* P) {
  if (P->g_chi0) return GW_OK;
  const long long slot = (long long)P->N * P->N * P->nw;
  const double per_q = 3.0 * sizeof(c128) * (double)slot;
  P->qb = (int)std::max(1.0, std::min((double)P->NK, std::floor(P->group_budget / per_q)));
  GW_TRY(dalloc(P, &P->g_chi0, (size_t)slot * P->qb));
  GW_TRY(dalloc(P, &P->g_E, (size_t)slot * P->qb));
  GW_TRY(dalloc(P, &P->g_work, (size_t)slot * P->qb));
  return GW_OK;
}

// The q loop of gw_g0w0 over the listed q points: groups of up to qb points whose FP64
// factorisations of eps~ run as one batched launch; Sigma_c terms accumulated into sig.
// -q on the mesh
int minus_q(const gw_plan_s* P, int q) {
  const int* n = P->p.nk;
  const int i3 = q % n[2], i2 = (q / n[2]) % n[1], i1 = q / (n[1] * n[2]);
  return (((n[0] - i1) % n[0]) * n[1] + (n[1] - i2) % n[1]) * n[2] + (n[2] - i3) % n[2];
}

// full: the list is the whole q mesh (then, with time reversal and no q -> 0 direction, only the
// target k <= -k are computed and the others copied: Sigma_c(-k) = Sigma_c(k))
gw_status g0w0_qlist(gw_plan_s* P, const std::vector<int>& qs_in, c128* sig_out, bool full = false) {
  cudaStream_t st = P->st;
  const int N = P->N, nw = P->nw;
  const long long NN = (long long)N * N;
  const long long slot = NN * nw;
  // time reversal: W^c(-q) = conj(W^c(q)), so of a pair (q, -q) in the list only the smaller q
  // goes through chi0 / eps~ / W^c; its W^c also gives the Sigma_c term of -q
  std::vector<int> qs, partner;
  {
    std::vector<char> in(P->NK, 0);
    for (int q : qs_in) in[q] = 1;
    for (int q : qs_in) {
      const int mq = P->trs ? minus_q(P, q) : q;
      if (mq != q && in[mq] && mq < q) continue;
      qs.push_back(q);
      partner.push_back(mq != q && in[mq] ? mq : -1);
    }
  }
  const bool halve_k = full && P->d_ktab;
  c128* sig = sig_out;
  if (halve_k) {
    sig = P->d_sigtmp;
    GW_CUDA(cudaMemsetAsync(sig, 0, sizeof(c128) * (size_t)P->NK * P->nsig * nw, st));
  }
  P->reset_timing();
  for (size_t g0 = 0; g0 < qs.size(); g0 += P->qb) {
    const int nq = (int)std::min<size_t>(P->qb, qs.size() - g0);
    const int* q = qs.data() + g0;
    const int* qp = partner.data() + g0;
    GW_CUDA(cudaMemsetAsync(P->d_status, 0, sizeof(int), st));
    GW_TRY(chi0_prepare(P, q, nq));
    for (int j = 0; j < nq; ++j) GW_TRY(chi0_core(P, q[j], P->g_chi0 + j * slot));
    for (int j = 0; j < nq; ++j) GW_TRY(eps_core(P, q[j], P->g_chi0 + j * slot, P->g_E + j * slot));
    launch_chol_inv_minus_I(N, P->g_E, nq * nw, NN, P->g_work, P->d_status, st);
    for (int j = 0; j < nq; ++j)
      if (q[j] == 0 && P->p.head_wings == 2) GW_TRY(q0_average(P, P->g_E + j * slot));
    for (int j = 0; j < nq; ++j) GW_TRY(w_core(P, q[j], P->g_E + j * slot, P->g_chi0 + j * slot));
    for (int j = 0; j < nq; ++j) {
      GW_TRY(sigma_core(P, q[j], P->g_chi0 + j * slot, sig, false, 0, -1, halve_k));
      if (qp[j] >= 0) GW_TRY(sigma_core(P, qp[j], P->g_chi0 + j * slot, sig, true, 0, -1, halve_k));
    }
    GW_TRY(read_status(P, "gw_g0w0"));
  }
  if (halve_k) {
    launch_sigma_trs_fill(P->NK, P->nsig, nw, P->p.nk, P->d_isrep, sig, sig_out, st);
    GW_TRY(check_launch(P, "Sigma_c time-reversal fill"));
  }
  GW_TRY(P->collect_timing());
  P->chi0_q = P->wc_q = -1;
  return GW_OK;
}

}  // namespace

extern "C" {

gw_status gw_chi0(gw_plan P, int32_t sys, int32_t q, gw_complex* chi0_out) {
  gw_status s;
  Route rt;
  if (!route(P, sys, rt, &s)) return s;
  if (!plan_ok(P, sys, &s)) return s;
  if (q < 0 || q >= P->NK) return fail(GW_ERR_ARG, "q out of range");
  cudaStream_t st = P->st;
  const size_t n = (size_t)P->N * P->N * P->nw;
  P->reset_timing();
  GW_CUDA(cudaMemsetAsync(P->d_status, 0, sizeof(int), st));
  GW_TRY(chi0_core(P, q, P->d_chi0));
  GW_TRY(read_status(P, "gw_chi0"));
  GW_TRY(P->collect_timing());
  if (chi0_out) GW_CUDA(cudaMemcpyAsync(chi0_out, P->d_chi0, sizeof(c128) * n, cudaMemcpyDeviceToDevice, st));
  P->chi0_q = q;
  P->wc_q = -1;
  return GW_OK;
}

gw_status gw_screen(gw_plan P, int32_t sys, int32_t q, gw_complex* wc_out) {
  gw_status s;
  Route rt;
  if (!route(P, sys, rt, &s)) return s;
  if (!plan_ok(P, sys, &s)) return s;
  if (q < 0 || q >= P->NK) return fail(GW_ERR_ARG, "q out of range");
  if (P->chi0_q != q) return fail(GW_ERR_STATE, "gw_screen needs gw_chi0 for the same q first");
  cudaStream_t st = P->st;
  const long long NN = (long long)P->N * P->N;
  GW_TRY(eps_core(P, q, P->d_chi0, P->d_E));
  GW_CUDA(cudaMemsetAsync(P->d_status, 0, sizeof(int), st));
  launch_chol_inv_minus_I(P->N, P->d_E, P->nw, NN, P->d_work, P->d_status, st);
  if (q == 0 && P->p.head_wings == 2) GW_TRY(q0_average(P, P->d_E));
  GW_TRY(w_core(P, q, P->d_E, P->d_Wc));
  GW_TRY(read_status(P, "gw_screen"));
  if (wc_out) GW_CUDA(cudaMemcpyAsync(wc_out, P->d_Wc, sizeof(c128) * NN * P->nw, cudaMemcpyDeviceToDevice, st));
  P->wc_q = q;
  return GW_OK;
}

gw_status gw_sigma(gw_plan P, int32_t sys, int32_t q, gw_complex* sigma_acc) {
  gw_status s;
  Route rt;
  if (!route(P, sys, rt, &s)) return s;
  if (!plan_ok(P, sys, &s)) return s;
  if (q < 0 || q >= P->NK) return fail(GW_ERR_ARG, "q out of range");
  if (P->wc_q != q) return fail(GW_ERR_STATE, "gw_sigma needs gw_screen for the same q first");
  c128* sig = sigma_acc ? reinterpret_cast<c128*>(sigma_acc) : P->d_sigma;
  GW_TRY(sigma_core(P, q, P->d_Wc, sig));
  return GW_OK;
}

gw_status gw_sigma_ext(gw_plan P, int32_t sys, int32_t q, const gw_complex* wc, int32_t k_lo, int32_t k_hi,
                       gw_complex* sigma_acc) {
  gw_status s;
  Route rt;
  if (!route(P, sys, rt, &s)) return s;
  if (!plan_ok(P, sys, &s)) return s;
  if (q < 0 || q >= P->NK) return fail(GW_ERR_ARG, "q out of range");
  if (!wc) return fail(GW_ERR_ARG, "wc is NULL");
  if (k_lo < 0 || k_hi > P->NK || k_lo >= k_hi) return fail(GW_ERR_ARG, "k range must satisfy 0 <= k_lo < k_hi <= N_k");
  c128* sig = sigma_acc ? reinterpret_cast<c128*>(sigma_acc) : P->d_sigma;
  GW_TRY(sigma_core(P, q, reinterpret_cast<const c128*>(wc), sig, false, k_lo, k_hi));
  return GW_OK;
}

gw_status gw_g0w0(gw_plan P, int32_t sys, gw_complex* sigma_acc) {
  gw_status s;
  Route rt;
  if (!route(P, sys, rt, &s)) return s;
  if (!plan_ok(P, sys, &s)) return s;
  if (P->sur.on && P->sur.model)
    return g0w0_sur(P, sigma_acc ? reinterpret_cast<c128*>(sigma_acc) : P->d_sigma);
  GW_TRY(ensure_groups(P));
  c128* sig = sigma_acc ? reinterpret_cast<c128*>(sigma_acc) : P->d_sigma;
  std::vector<int> qs(P->NK);
  for (int q = 0; q < P->NK; ++q) qs[q] = q;
  return g0w0_qlist(P, qs, sig, true);
}

gw_status gw_g0w0_qset(gw_plan P, int32_t sys, const int32_t* q_list, int32_t n_q, gw_complex* sigma_acc) {
  gw_status s;
  Route rt;
  if (!route(P, sys, rt, &s)) return s;
  if (!plan_ok(P, sys, &s)) return s;
  if (n_q < 0 || (n_q > 0 && !q_list)) return fail(GW_ERR_ARG, "q_list is NULL or n_q < 0");
  if (!sigma_acc) return fail(GW_ERR_ARG, "sigma_acc is NULL");
  if (P->sur.on && P->sur.model) return fail(GW_ERR_UNSUPPORTED, "gw_g0w0_qset: a surrogate is attached");
  std::vector<int> qs(q_list, q_list + n_q);
  std::vector<char> seen(P->NK, 0);
  for (int q : qs) {
    if (q < 0 || q >= P->NK) return fail(GW_ERR_ARG, "gw_g0w0_qset: q out of range");
    if (seen[q]++) return fail(GW_ERR_ARG, "gw_g0w0_qset: q listed twice");
  }
  GW_TRY(ensure_groups(P));
  return g0w0_qlist(P, qs, reinterpret_cast<c128*>(sigma_acc));
}

gw_status gw_qp(gw_plan P, int32_t sys, const gw_complex* sigma, const double* dxv, double* e_qp, double* gap,
                int32_t* n_conv) {
  gw_status s;
  Route rt;
  if (!route(P, sys, rt, &s)) return s;
  if (!plan_ok(P, sys, &s)) return s;
  if (!e_qp || !gap) return fail(GW_ERR_ARG, "e_qp and gap must not be NULL");
  cudaStream_t st = P->st;
  const int n = P->NK * P->nsig;
  double* d_e;
  int* d_c;
  GW_TRY(dalloc(P, &d_e, n));
  GW_TRY(dalloc(P, &d_c, n));
  const c128* sg = sigma ? reinterpret_cast<const c128*>(sigma) : P->d_sigma;
  launch_qp(P->NK, P->nsig, P->NBd, P->p.sigma_lo, P->nw, sg, dxv, P->p.eps, P->d_mu, P->d_freq, d_e, d_c, st);
  GW_TRY(check_launch(P, "gw_qp"));
  std::vector<int> conv(n);
  GW_CUDA(cudaMemcpyAsync(e_qp, d_e, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  GW_CUDA(cudaMemcpyAsync(conv.data(), d_c, n * sizeof(int), cudaMemcpyDeviceToHost, st));
  GW_CUDA(cudaStreamSynchronize(st));
  dfree_last(P);
  dfree_last(P);
  int nc = 0;
  for (int i = 0; i < n; ++i) nc += conv[i];
  if (n_conv) *n_conv = nc;
  const int h = P->nocc - 1 - P->p.sigma_lo, l = P->nocc - P->p.sigma_lo;
  if (h >= 0 && h < P->nsig && l >= 0 && l < P->nsig) {
    double hmax = -1e300, lmin = 1e300;
    for (int k = 0; k < P->NK; ++k) {
      hmax = std::max(hmax, e_qp[k * P->nsig + h]);
      lmin = std::min(lmin, e_qp[k * P->nsig + l]);
    }
    *gap = lmin - hmax;
  } else {
    *gap = std::nan("");
  }
  return GW_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// gw_qp_static: the QP solve of gw_qp with its device scratch (per-(k, n) energies and Newton
// flags) in one fixed file-scope array instead of a cudaMalloc/cudaFree pair per call.
// Callers that cannot allocate at that point use it: a process whose device memory is held by
// a caching allocator (the pool is full, so a fresh cudaMalloc fails although the QP step
// needs only a few hundred KB), and a serving loop that re-solves the QP equation after every
// Sigma_c update and cannot take the device-wide synchronisation that cudaFree implies.
// The paper has no counterpart: it is a deployment variant of the QP step.
// ---------------------------------------------------------------------------------------------
#include <mutex>

namespace {

struct QpScratch {
  double e_qp[GW_QP_STATIC_MAX];  // written for every (k, n) < N_k * n_sigma by k_qp
  int conv[GW_QP_STATIC_MAX];     // written for every (k, n) < N_k * n_sigma by k_qp
  int n_conv;                     // written by k_qp_count
};
// Nothing here has to start at zero: each call writes every element it later reads.
static __device__ __align__(256) QpScratch g_qp_scratch;

std::mutex g_qp_scratch_mu;
QpScratch* g_qp_scratch_ptr[64] = {};  // per device ordinal, looked up on the first call there

// Device address of g_qp_scratch on the current device. The first call on a device makes the
// lookup (cudaGetSymbolAddress, which may load this module onto the device).
gw_status qp_scratch(QpScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(GW_ERR_CUDA, std::string("gw_qp_static: cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return fail(GW_ERR_UNSUPPORTED, "gw_qp_static: device ordinal above 63");
  std::lock_guard<std::mutex> lk(g_qp_scratch_mu);
  if (!g_qp_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_qp_scratch);
    if (e != cudaSuccess || p == nullptr)
      return fail(GW_ERR_CUDA, std::string("gw_qp_static: cudaGetSymbolAddress of the scratch array: ") +
                                   cudaGetErrorString(e));
    g_qp_scratch_ptr[dev] = static_cast<QpScratch*>(p);
  }
  *out = g_qp_scratch_ptr[dev];
  return GW_OK;
}

// Number of converged (k, n) pairs: one block sums the flags.
__global__ void k_qp_count(const int* __restrict__ conv, int n, int* out) {
  __shared__ int s[256];
  int acc = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += conv[i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

}  // namespace

extern "C" {

gw_status gw_qp_static(gw_plan P, int32_t sys, const gw_complex* sigma, const double* dxv, double* e_qp,
                       double* gap, int32_t* n_conv) {
  gw_status s;
  Route rt;
  if (!route(P, sys, rt, &s)) return s;
  if (!plan_ok(P, sys, &s)) return s;
  if (!e_qp || !gap) return fail(GW_ERR_ARG, "e_qp and gap must not be NULL");
  const int n = P->NK * P->nsig;
  if (n > GW_QP_STATIC_MAX)
    return fail(GW_ERR_ARG, "gw_qp_static: N_k * n_sigma = " + std::to_string(n) +
                                " exceeds the static scratch capacity GW_QP_STATIC_MAX = " +
                                std::to_string(GW_QP_STATIC_MAX) + "; use gw_qp");
  int cur = -1;
  GW_CUDA(cudaGetDevice(&cur));
  if (cur != P->dev)
    return fail(GW_ERR_STATE, "gw_qp_static: the current device (" + std::to_string(cur) +
                                  ") is not the plan's device (" + std::to_string(P->dev) + ")");
  QpScratch* sc = nullptr;
  GW_TRY(qp_scratch(&sc));
  cudaStream_t st = P->st;
  const c128* sg = sigma ? reinterpret_cast<const c128*>(sigma) : P->d_sigma;
  launch_qp(P->NK, P->nsig, P->NBd, P->p.sigma_lo, P->nw, sg, dxv, P->p.eps, P->d_mu, P->d_freq, sc->e_qp, sc->conv,
            st);
  GW_TRY(check_launch(P, "gw_qp_static"));
  ++g_launch_count, k_qp_count<<<1, 256, 0, st>>>(sc->conv, n, &sc->n_conv);
  GW_TRY(check_launch(P, "gw_qp_static"));
  int nc = 0;
  GW_CUDA(cudaMemcpyAsync(e_qp, sc->e_qp, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st));
  GW_CUDA(cudaMemcpyAsync(&nc, &sc->n_conv, sizeof(int), cudaMemcpyDeviceToHost, st));
  GW_CUDA(cudaStreamSynchronize(st));
  if (n_conv) *n_conv = nc;
  const int h = P->nocc - 1 - P->p.sigma_lo, l = P->nocc - P->p.sigma_lo;
  if (h >= 0 && h < P->nsig && l >= 0 && l < P->nsig) {
    double hmax = -1e300, lmin = 1e300;
    for (int k = 0; k < P->NK; ++k) {
      hmax = std::max(hmax, e_qp[k * P->nsig + h]);
      lmin = std::min(lmin, e_qp[k * P->nsig + l]);
    }
    *gap = lmin - hmax;
  } else {
    *gap = std::nan("");
  }
  return GW_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Learned frequency surrogate on the plan (the paper has no counterpart): chi0 / eps~ only on
// the coarse frequencies C, X = eps~^-1 - 1 on the fine frequencies F from
//   X(w_m) = sum_c L_mc X(w_c) + U diag(sigma_l g_l(w_m)) U^H,
// U the Ritz modes of eps~(w_ref) - 1. Sigma_c needs only S_nm(w') = a^T V^1/2 X V^1/2 a^*,
// which is linear in X:  S(w_m) = sum_c L_mc S(w_c) + sum_l |p_l|^2 sigma_l g_l(w_m),
// p = a^T (V^1/2 U). So the W^c contraction runs on the coarse frequencies only, plus one
// projection of the rows a onto V^1/2 U.
// ---------------------------------------------------------------------------------------------
namespace {

// plan views of the frequency grid: nw and d_freq replaced while alive
struct FreqView {
  gw_plan_s* P;
  int nw;
  double* freq;
  FreqView(gw_plan_s* P_, int nw_, double* f_) : P(P_), nw(P_->nw), freq(P_->d_freq) {
    P->nw = nw_;
    P->d_freq = f_;
  }
  ~FreqView() {
    P->nw = nw;
    P->d_freq = freq;
  }
};

// batch buffers of the mode computation for up to cap problems (grown, never shrunk)
gw_status sur_ensure_batch(gw_plan_s* P, int cap) {
  SurState& S = P->sur;
  if (cap <= S.bcap) return GW_OK;
  const size_t N = P->N, nb = S.nb, c = cap;
  GW_TRY(dalloc(P, &S.d_Y, c * N * nb));
  GW_TRY(dalloc(P, &S.d_Q, c * N * nb));
  GW_TRY(dalloc(P, &S.d_T, c * N * nb));
  GW_TRY(dalloc(P, &S.d_G, c * nb * nb));
  GW_TRY(dalloc(P, &S.d_Linv, c * nb * nb));
  GW_TRY(dalloc(P, &S.d_H, c * nb * nb));
  GW_TRY(dalloc(P, &S.d_Z, c * nb * nb));
  GW_TRY(dalloc(P, &S.d_theta, c * nb));
  S.bcap = cap;
  return GW_OK;
}

// Q_j = orth(Y_j), j < nq, by two Cholesky-QR passes (Y and T are overwritten)
void cholqr2(gw_plan_s* P, int nq, c128* Y, c128* Q) {
  SurState& S = P->sur;
  const int N = P->N, nb = S.nb;
  const long long sY = (long long)N * nb, sG = (long long)nb * nb;
  const c128 one{1, 0}, zero{0, 0};
  c128* in = Y;
  c128* outs[2] = {S.d_T, Q};
  for (int pass = 0; pass < 2; ++pass) {
    launch_zgemm<double>(nb, nb, N, one, in, nb, sY, OP_C, in, nb, sY, OP_N, zero, S.d_G, nb, sG, nq, P->st);
    launch_small_chol_linv(nb, nq, S.d_G, S.d_Linv, P->d_status, P->st);
    launch_zgemm<double>(N, nb, nb, one, in, nb, sY, OP_N, S.d_Linv, nb, sG, OP_C, zero, outs[pass], nb, sY, nq, P->st);
    in = outs[pass];
  }
}

// Ritz modes of nq Hermitian matrices A_j = A + j*sA [N][N]: subspace iteration from the start
// block, Rayleigh-Ritz; U_j = U + j*sU [N][k] = the k Ritz vectors of largest Ritz value
// (S.d_theta + j*nb holds all nb Ritz values of problem j, descending)
gw_status modes_core(gw_plan_s* P, const c128* A, long long sA, int nq, c128* U, long long sU) {
  SurState& S = P->sur;
  const int N = P->N, nb = S.nb, k = S.k;
  const long long sY = (long long)N * nb, sG = (long long)nb * nb;
  const c128 one{1, 0}, zero{0, 0};
  cudaStream_t st = P->st;
  GW_TRY(sur_ensure_batch(P, nq));
  for (int j = 0; j < nq; ++j)
    GW_CUDA(cudaMemcpyAsync(S.d_Y + j * sY, S.d_start, sizeof(c128) * sY, cudaMemcpyDeviceToDevice, st));
  cholqr2(P, nq, S.d_Y, S.d_Q);
  for (int it = 0; it < S.iters; ++it) {
    launch_zgemm<double>(N, nb, N, one, A, N, sA, OP_N, S.d_Q, nb, sY, OP_N, zero, S.d_Y, nb, sY, nq, st);
    cholqr2(P, nq, S.d_Y, S.d_Q);
  }
  launch_zgemm<double>(N, nb, N, one, A, N, sA, OP_N, S.d_Q, nb, sY, OP_N, zero, S.d_Y, nb, sY, nq, st);
  launch_zgemm<double>(nb, nb, N, one, S.d_Q, nb, sY, OP_C, S.d_Y, nb, sY, OP_N, zero, S.d_H, nb, sG, nq, st);
  launch_small_jacobi(nb, nq, S.d_H, S.d_theta, S.d_Z, st);
  launch_zgemm<double>(N, k, nb, one, S.d_Q, nb, sY, OP_N, S.d_Z, nb, sG, OP_N, zero, U, k, sU, nq, st);
  return check_launch(P, "surrogate modes");
}

// d rows j*k .. (j+1)*k-1, columns 0 .. nx-1 (leading dimension ldd): mode diagonal of the nx
// matrices X + j*sX [nx][N][N] in the basis U + j*sU, for j < nq
void mode_diag(gw_plan_s* P, const c128* X, long long sX, int nx, int nq, const c128* U, long long sU, float* d,
               int ldd) {
  SurState& S = P->sur;
  const int N = P->N, k = S.k;
  const long long NN = (long long)N * N;
  const c128 one{1, 0}, zero{0, 0};
  for (int j = 0; j < nq; ++j) {
    const c128* Uj = U + j * sU;
    launch_zgemm<double>(N, k, N, one, X + j * sX, N, NN, OP_N, Uj, k, 0, OP_N, zero, S.d_XU, k, (long long)N * k, nx,
                         P->st);
    launch_mode_diag(N, k, nx, Uj, S.d_XU, (long long)N * k, d + (long long)j * k * ldd, ldd, 0, P->st);
  }
}

// q term of Sigma_c with W^c on the coarse frequencies (Wc_c [nc][N][N]), the modes U [N][k]
// and the network's correction coef [k][nf] (sigma_l g_l(w_m)); full-grid convolution.
gw_status sigma_core_sur(gw_plan_s* P, int q, const c128* Wc_c, const c128* U, const float* coef, c128* sig) {
  SurState& S = P->sur;
  cudaStream_t st = P->st;
  const int N = P->N, nw = P->nw, nc = S.nc, nf = S.nf, k = S.k, NBd = P->NBd, nsig = P->nsig;
  const long long NN = (long long)N * N;
  const c128* evec = reinterpret_cast<const c128*>(P->p.evec);
  const double pref = -1.0 / (2.0 * M_PI * P->NK);
  const int tf32 = P->prec == GW_3XTF32;
  const float* Lmat = sur_linear(S.model);
  // B = V^1/2 U
  launch_zgemm<double>(N, k, N, c128{1, 0}, P->d_Vh + (long long)q * NN, N, 0, OP_N, U, k, 0, OP_N, c128{0, 0}, S.d_B,
                       k, 0, 1, st);
  c64* B32 = reinterpret_cast<c64*>(S.d_XU);
  if (!P->fp64) {
    launch_convert(N * k, S.d_B, B32, st);
    tc_w_planes(N, nc, P->Kx, Wc_c, P->d_Wpl, tf32, st);
  }
  for (int kk0 = 0; kk0 < P->NK; kk0 += P->sig_nkk) {
    const int nkk = std::min(P->sig_nkk, P->NK - kk0);
    const int R = nkk * nsig * NBd;
    if (P->fp64) {
      c128* A = static_cast<c128*>(P->d_A);
      c128* Ut = static_cast<c128*>(P->d_U);
      launch_mgen<double>(P->geom, static_cast<const c128*>(P->d_T1), nullptr, evec, q, kk0, nkk,
                          MAP_K_IS_KK_MINUS_Q, P->p.sigma_lo, nsig, 0, NBd, A, N, 1, st);
      for (int c = 0; c < nc; ++c) {
        launch_zgemm<double>(R, N, N, c128{1, 0}, A, N, 0, OP_N, Wc_c + c * NN, N, 0, OP_N, c128{0, 0}, Ut, N, 0, 1, st);
        launch_rowdot<double>(R, N, Ut, A, N, nullptr, S.d_Sc_d, c, nc, st);
      }
      c128* Pm = static_cast<c128*>(S.d_P);
      launch_zgemm<double>(R, k, N, c128{1, 0}, A, N, 0, OP_N, S.d_B, k, 0, OP_N, c128{0, 0}, Pm, k, 0, 1, st);
      launch_sur_assemble<double>(R, nc, nw, k, S.d_jmap, S.d_Sc_d, Pm, coef, nf, Lmat, P->d_S_d, st);
    } else {
      c64* A = static_cast<c64*>(P->d_A);
      if (!launch_mgen_sig(P->geom, static_cast<const c64*>(P->d_T1), evec, q, kk0, nkk, P->p.sigma_lo, nsig, NBd,
                           A, P->Kx, 1, st) &&
          !P->mtune.run(0, nsig, NBd, st, [&](int v) {
            launch_mgen<float>(P->geom, static_cast<const c64*>(P->d_T1), nullptr, evec, q, kk0, nkk,
                               MAP_K_IS_KK_MINUS_Q, P->p.sigma_lo, nsig, 0, NBd, A, P->Kx, 1, st, v);
          }))
        return fail(GW_ERR_CUDA, "M kernel autotuner: CUDA error");
      GW_CUDA(cudaMemsetAsync(S.d_Sc, 0, sizeof(float) * (size_t)R * nc, st));
      TcSigmaArgs a{};
      a.R = R;
      a.N = N;
      a.Kpad = P->Kx;
      a.nw = nc;
      a.raw = reinterpret_cast<const float*>(A);
      for (int i = 0; i < 6; ++i) a.bpl[i] = P->d_Wpl.b[i];
      a.S = S.d_Sc;
      a.apl[0] = P->d_Apl[0];
      a.apl[1] = P->d_Apl[1];
      a.tf32 = tf32;
      a.status = P->d_status;
      std::string err;
      gw_status ts = tc_sigma_run(a, st, err);
      if (ts != GW_OK) {
        P->err = 1;
        return fail(ts, err);
      }
      c64* Pm = static_cast<c64*>(S.d_P);
      launch_zgemm<float>(R, k, N, c64{1, 0}, A, P->Kx, 0, OP_N, B32, k, 0, OP_N, c64{0, 0}, Pm, k, 0, 1, st);
      launch_sur_assemble<float>(R, nc, nw, k, S.d_jmap, S.d_Sc, Pm, coef, nf, Lmat, P->d_S_f, st);
    }
    launch_sigma_conv_chunk(kk0, nkk, nsig, NBd, P->p.nk, q, P->p.eps, P->d_mu, P->d_S_f, P->d_S_d, P->d_freq,
                            P->d_fw, nw, pref, sig, P->fp64, st);
    GW_TRY(check_launch(P, "Sigma_c (surrogate)"));
  }
  return GW_OK;
}

// the whole q loop with the surrogate: q groups as gw_g0w0, coarse frequencies only
gw_status g0w0_sur(gw_plan_s* P, c128* sig) {
  SurState& S = P->sur;
  cudaStream_t st = P->st;
  const int N = P->N, nc = S.nc, nf = S.nf, k = S.k;
  const long long NN = (long long)N * N;
  const long long slot = NN * nc;
  if (!S.g_chi0) {
    const double per_q = 3.0 * sizeof(c128) * (double)slot + sizeof(c128) * (double)(NN + (long long)N * k);
    S.qbs = (int)std::max(1.0, std::min({(double)P->NK, std::floor(6.0e9 / per_q), std::floor(4096.0 / k)}));
    GW_TRY(dalloc(P, &S.g_chi0, (size_t)slot * S.qbs));
    GW_TRY(dalloc(P, &S.g_E, (size_t)slot * S.qbs));
    GW_TRY(dalloc(P, &S.g_work, (size_t)slot * S.qbs));
    GW_TRY(dalloc(P, &S.g_A, (size_t)NN * S.qbs));
    GW_TRY(dalloc(P, &S.g_U, (size_t)N * k * S.qbs));
    const size_t rows = (size_t)S.qbs * k;
    GW_TRY(dalloc(P, &S.d_d, rows * nc));
    GW_TRY(dalloc(P, &S.d_x, rows * nc));
    GW_TRY(dalloc(P, &S.d_sig, rows));
    GW_TRY(dalloc(P, &S.d_g, rows * nf));
    GW_TRY(dalloc(P, &S.d_coef, rows * nf));
  }
  P->reset_timing();
  for (int q0 = 0; q0 < P->NK; q0 += S.qbs) {
    const int nq = std::min(S.qbs, P->NK - q0);
    GW_CUDA(cudaMemsetAsync(P->d_status, 0, sizeof(int), st));
    {
      FreqView fv(P, nc, S.d_freq_c);
      std::vector<int> qg(nq);
      for (int j = 0; j < nq; ++j) qg[j] = q0 + j;
      GW_TRY(chi0_prepare(P, qg.data(), nq));
      for (int j = 0; j < nq; ++j) GW_TRY(chi0_core(P, q0 + j, S.g_chi0 + j * slot));
      for (int j = 0; j < nq; ++j) {
        GW_TRY(eps_core(P, q0 + j, S.g_chi0 + j * slot, S.g_E + j * slot));
        GW_CUDA(cudaMemcpyAsync(S.g_A + j * NN, S.g_E + j * slot, sizeof(c128) * NN, cudaMemcpyDeviceToDevice, st));
      }
      launch_axpby_identity<double>(N, S.g_A, NN, nq, -1.0, st);
      launch_chol_inv_minus_I(N, S.g_E, nq * nc, NN, S.g_work, P->d_status, st);
      GW_TRY(modes_core(P, S.g_A, NN, nq, S.g_U, (long long)N * k));
      mode_diag(P, S.g_E, slot, nc, nq, S.g_U, (long long)N * k, S.d_d, nc);
      launch_sur_inputs(nq * k, nc, S.d_d, S.d_x, S.d_sig, st);
      GW_TRY(sur_correction(S.model, S.d_x, nq * k, S.d_g, st));
      launch_sur_coef(nq * k, nf, S.d_sig, S.d_g, S.d_coef, st);
      for (int j = 0; j < nq; ++j) GW_TRY(w_core(P, q0 + j, S.g_E + j * slot, S.g_chi0 + j * slot));
    }
    for (int j = 0; j < nq; ++j)
      GW_TRY(sigma_core_sur(P, q0 + j, S.g_chi0 + j * slot, S.g_U + (long long)j * N * k,
                            S.d_coef + (long long)j * k * nf, sig));
    GW_TRY(read_status(P, "gw_g0w0 (surrogate)"));
  }
  GW_TRY(P->collect_timing());
  P->chi0_q = P->wc_q = -1;
  return GW_OK;
}

}  // namespace

extern "C" {

gw_status gw_surrogate_enable(gw_plan P, gw_surrogate model, const gw_surrogate_cfg* cfg) {
  gw_status s;
  if (P && !P->subs.empty()) return fail(GW_ERR_UNSUPPORTED, "gw_surrogate_enable: not on a batch plan");
  if (!plan_ok(P, 0, &s)) return s;
  if (P->p.head_wings == 2 && cfg)
    return fail(GW_ERR_UNSUPPORTED, "gw_surrogate_enable: not with the direction-averaged q = 0 (head_wings = 2)");
  SurState& S = P->sur;
  if (!cfg) {
    if (model) return fail(GW_ERR_ARG, "gw_surrogate_enable: a model needs a configuration");
    S.on = false;
    S.model = nullptr;
    return GW_OK;
  }
  const int N = P->N, nw = P->nw;
  const int nc = cfg->n_coarse, k = cfg->n_modes, nb = cfg->n_block;
  if (nc < 1 || nc > nw || nc > 64 || !cfg->coarse) return fail(GW_ERR_ARG, "gw_surrogate_enable: bad n_coarse / coarse");
  for (int i = 0; i < nc; ++i) {
    if (cfg->coarse[i] < 0 || cfg->coarse[i] >= nw || (i && cfg->coarse[i] <= cfg->coarse[i - 1]))
      return fail(GW_ERR_ARG, "gw_surrogate_enable: coarse indices must be ascending grid indices");
  }
  if (nb < 1 || nb > 64 || nb > N || k < 1 || k > nb) return fail(GW_ERR_ARG, "gw_surrogate_enable: need 1 <= n_modes <= n_block <= min(64, n_aux)");
  if (cfg->n_iter < 0 || cfg->n_iter > 1000 || !cfg->start) return fail(GW_ERR_ARG, "gw_surrogate_enable: bad n_iter or start");
  if (model && (sur_n_in(model) != nc || sur_n_out(model) != nw - nc))
    return fail(GW_ERR_ARG, "gw_surrogate_enable: the model's n_in / n_out must be n_coarse / n_freq - n_coarse");
  if (S.d_jmap && (S.nc != nc || S.k != k || S.nb != nb))
    return fail(GW_ERR_UNSUPPORTED, "gw_surrogate_enable: sizes cannot change once set on a plan");
  cudaStream_t st = P->st;
  S.coarse.assign(cfg->coarse, cfg->coarse + nc);
  S.fine.clear();
  std::vector<int> jmap(nw);
  for (int j = 0, c = 0; j < nw; ++j) {
    if (c < nc && S.coarse[c] == j) {
      jmap[j] = c++;
    } else {
      jmap[j] = -(int)S.fine.size() - 1;
      S.fine.push_back(j);
    }
  }
  S.nc = nc;
  S.nf = nw - nc;
  S.k = k;
  S.nb = nb;
  S.iters = cfg->n_iter;
  if (!S.d_jmap) {
    const size_t rows = (size_t)P->sig_rows;
    GW_TRY(dalloc(P, &S.d_jmap, nw));
    GW_TRY(dalloc(P, &S.d_cidx, nw));
    GW_TRY(dalloc(P, &S.d_fidx, nw));
    GW_TRY(dalloc(P, &S.d_freq_c, nc));
    GW_TRY(dalloc(P, &S.d_start, (size_t)N * nb));
    GW_TRY(sur_ensure_batch(P, 1));
    GW_TRY(dalloc(P, &S.d_A1, (size_t)N * N));
    GW_TRY(dalloc(P, &S.d_U1, (size_t)N * k));
    GW_TRY(dalloc(P, &S.d_XU, (size_t)std::max(nw, nc) * N * k));
    GW_TRY(dalloc(P, &S.d_B, (size_t)N * k));
    c128* pp = nullptr;
    GW_TRY(dalloc(P, &pp, rows * k));
    S.d_P = pp;
    GW_TRY(dalloc(P, &S.d_Sc, rows * nc));
    GW_TRY(dalloc(P, &S.d_Sc_d, rows * nc));
  }
  std::vector<double> fc(nc);
  for (int i = 0; i < nc; ++i) fc[i] = P->freq[S.coarse[i]];
  GW_CUDA(cudaMemcpyAsync(S.d_jmap, jmap.data(), sizeof(int) * nw, cudaMemcpyHostToDevice, st));
  GW_CUDA(cudaMemcpyAsync(S.d_cidx, S.coarse.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, st));
  if (!S.fine.empty())
    GW_CUDA(cudaMemcpyAsync(S.d_fidx, S.fine.data(), sizeof(int) * S.fine.size(), cudaMemcpyHostToDevice, st));
  GW_CUDA(cudaMemcpyAsync(S.d_freq_c, fc.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, st));
  GW_CUDA(cudaMemcpyAsync(S.d_start, cfg->start, sizeof(c128) * N * nb, cudaMemcpyDeviceToDevice, st));
  GW_CUDA(cudaStreamSynchronize(st));
  S.model = model;
  S.on = true;
  return GW_OK;
}

gw_status gw_surrogate_modes(gw_plan P, int32_t sys, int32_t q, float* d_out, double* theta_out, float* x_out,
                             float* y_out) {
  gw_status s;
  Route rt;
  if (!route(P, sys, rt, &s)) return s;
  if (!plan_ok(P, sys, &s)) return s;
  SurState& S = P->sur;
  if (!S.on) return fail(GW_ERR_STATE, "gw_surrogate_modes needs gw_surrogate_enable first");
  if (q < 0 || q >= P->NK || (!d_out && !x_out && !y_out)) return fail(GW_ERR_ARG, "gw_surrogate_modes: bad q or no output");
  if (y_out && S.nf < 1) return fail(GW_ERR_ARG, "gw_surrogate_modes: no fine frequencies for y_out");
  if (P->chi0_q != q) return fail(GW_ERR_STATE, "gw_surrogate_modes needs gw_chi0 for the same q first");
  cudaStream_t st = P->st;
  const int N = P->N, nw = P->nw;
  const long long NN = (long long)N * N;
  GW_CUDA(cudaMemsetAsync(P->d_status, 0, sizeof(int), st));
  GW_TRY(eps_core(P, q, P->d_chi0, P->d_E));
  GW_CUDA(cudaMemcpyAsync(S.d_A1, P->d_E + S.coarse[0] * NN, sizeof(c128) * NN, cudaMemcpyDeviceToDevice, st));
  launch_axpby_identity<double>(N, S.d_A1, NN, 1, -1.0, st);
  launch_chol_inv_minus_I(N, P->d_E, nw, NN, P->d_work, P->d_status, st);
  GW_TRY(modes_core(P, S.d_A1, 0, 1, S.d_U1, 0));
  float* d = d_out ? d_out : reinterpret_cast<float*>(P->d_tmp);
  mode_diag(P, P->d_E, 0, nw, 1, S.d_U1, 0, d, nw);
  if (x_out || y_out) launch_sur_features(S.k, nw, S.coarse[0], S.d_jmap, d, S.nc, S.nf, x_out, y_out, st);
  if (theta_out) GW_CUDA(cudaMemcpyAsync(theta_out, S.d_theta, sizeof(double) * S.k, cudaMemcpyDeviceToDevice, st));
  GW_TRY(check_launch(P, "gw_surrogate_modes"));
  return read_status(P, "gw_surrogate_modes");
}

}  // extern "C"

extern "C" {

gw_status gw_surrogate_data(gw_plan P, int32_t sys, float* x_out, float* y_out, double* moments) {
  gw_status s;
  Route rt;
  if (!route(P, sys, rt, &s)) return s;
  if (!plan_ok(P, sys, &s)) return s;
  SurState& S = P->sur;
  if (!S.on) return fail(GW_ERR_STATE, "gw_surrogate_data needs gw_surrogate_enable first");
  if (!x_out || !y_out || S.nf < 1) return fail(GW_ERR_ARG, "gw_surrogate_data: x_out / y_out NULL or no fine frequencies");
  if (moments && (P->nw > 64 || S.nc * P->nw > 1024))
    return fail(GW_ERR_UNSUPPORTED, "gw_surrogate_data: moments need n_freq <= 64 and n_coarse * n_freq <= 1024");
  cudaStream_t st = P->st;
  const int N = P->N, nw = P->nw, k = S.k;
  const long long NN = (long long)N * N, slot = NN * nw;
  GW_TRY(ensure_groups(P));
  if (!S.g_Af) {
    GW_TRY(dalloc(P, &S.g_Af, (size_t)NN * P->qb));
    GW_TRY(dalloc(P, &S.g_Uf, (size_t)N * k * P->qb));
    GW_TRY(dalloc(P, &S.d_df, (size_t)P->qb * k * nw));
  }
  P->reset_timing();
  for (int q0 = 0; q0 < P->NK; q0 += P->qb) {
    const int nq = std::min(P->qb, P->NK - q0);
    GW_CUDA(cudaMemsetAsync(P->d_status, 0, sizeof(int), st));
    std::vector<int> qg(nq);
    for (int j = 0; j < nq; ++j) qg[j] = q0 + j;
    GW_TRY(chi0_prepare(P, qg.data(), nq));
    for (int j = 0; j < nq; ++j) GW_TRY(chi0_core(P, q0 + j, P->g_chi0 + j * slot));
    for (int j = 0; j < nq; ++j) {
      GW_TRY(eps_core(P, q0 + j, P->g_chi0 + j * slot, P->g_E + j * slot));
      GW_CUDA(cudaMemcpyAsync(S.g_Af + j * NN, P->g_E + j * slot + S.coarse[0] * NN, sizeof(c128) * NN,
                              cudaMemcpyDeviceToDevice, st));
    }
    launch_axpby_identity<double>(N, S.g_Af, NN, nq, -1.0, st);
    launch_chol_inv_minus_I(N, P->g_E, nq * nw, NN, P->g_work, P->d_status, st);
    GW_TRY(modes_core(P, S.g_Af, NN, nq, S.g_Uf, (long long)N * k));
    mode_diag(P, P->g_E, slot, nw, nq, S.g_Uf, (long long)N * k, S.d_df, nw);
    if (moments)
      for (int j = 0; j < nq; ++j)
        launch_freq_moments(nw, NN, P->g_E + j * slot, S.d_cidx, S.d_fidx, S.nc, S.nf, moments, st);
    launch_sur_features(nq * k, nw, S.coarse[0], S.d_jmap, S.d_df, S.nc, S.nf, x_out + (long long)q0 * k * S.nc,
                        y_out + (long long)q0 * k * S.nf, st);
    GW_TRY(check_launch(P, "gw_surrogate_data"));
    GW_TRY(read_status(P, "gw_surrogate_data"));
  }
  GW_TRY(P->collect_timing());
  P->chi0_q = P->wc_q = -1;
  return GW_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Batch of independent systems (gw_plan_create with n_sys > 1): every system's whole q loop
// (gw_g0w0) on its own stream, driven by a pool of host threads, so that the kernels of
// different systems run concurrently and fill the GPU when single systems are small.
// ---------------------------------------------------------------------------------------------
#include <atomic>
#include <thread>

extern "C" {

gw_status gw_g0w0_batch(gw_plan P, gw_complex* const* sigma_accs, int32_t n_threads) {
  if (!P) return fail(GW_ERR_ARG, "plan is NULL");
  if (P->subs.empty()) return gw_g0w0(P, 0, sigma_accs ? sigma_accs[0] : nullptr);
  const int n = (int)P->subs.size();
  if (n_threads < 0) return fail(GW_ERR_ARG, "n_threads must be >= 0");
  const int nt = std::max(1, std::min(n, n_threads > 0 ? (int)n_threads : 8));
  GW_CUDA(cudaStreamSynchronize(P->st));
  int dev = 0;
  GW_CUDA(cudaGetDevice(&dev));
  std::vector<gw_status> st(n, GW_OK);
  std::vector<std::string> msg(n);
  std::atomic<int> next{0};
  auto worker = [&]() {
    cudaSetDevice(dev);
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= n) break;
      st[i] = gw_g0w0(P->subs[i], 0, sigma_accs ? sigma_accs[i] : nullptr);
      if (st[i] != GW_OK) msg[i] = gw_last_error();
      cudaStreamSynchronize(P->subs[i]->st);
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
  worker();
  for (auto& th : pool) th.join();
  for (int i = 0; i < n; ++i)
    if (st[i] != GW_OK) return fail(st[i], "system " + std::to_string(i) + ": " + msg[i]);
  return GW_OK;
}

gw_status gw_plan_n_sys(gw_plan P, int32_t* n_sys) {
  if (!P || !n_sys) return fail(GW_ERR_ARG, "NULL argument");
  *n_sys = P->subs.empty() ? 1 : (int32_t)P->subs.size();
  return GW_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Exchange self-energy (the bare-Coulomb part of Eq. GW_selfe_element, W = V + W^c):
//   Sigma_x_n(k) = -(1/N_q) sum_q sum_{m occ} a^T V(q) a^*,  a = C_{nm}(k, k-q) = M_{nm}(k-q, q)
// Rows a_r, r = ((kk * n_sigma) + n) * n_occ + m, as for Sigma_c but over the occupied bands;
// U = A V(q) (FP64 GEMM on the FP64 path, FP32 on the split paths), S_r = Re U_r . conj(a_r).
// ---------------------------------------------------------------------------------------------
namespace {

__global__ void k_sigx_accum(int nkk, int kk0, int nsig, int nocc, const double* __restrict__ S, double scale,
                             double* __restrict__ sigx) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nkk * nsig) return;
  double acc = 0.0;
  for (int m = 0; m < nocc; ++m) acc += S[(long long)e * nocc + m];
  sigx[(long long)kk0 * nsig + e] += scale * acc;
}

}  // namespace

extern "C" {

gw_status gw_sigma_x(gw_plan P, int32_t sys, double* sigx) {
  gw_status s;
  Route rt;
  if (!route(P, sys, rt, &s)) return s;
  if (!plan_ok(P, sys, &s)) return s;
  if (!sigx) return fail(GW_ERR_ARG, "gw_sigma_x: sigx is NULL");
  cudaStream_t st = P->st;
  const int N = P->N, nsig = P->nsig, nocc = P->nocc;
  const long long NN = (long long)N * N;
  const long long rows_max = (long long)P->sig_nkk * nsig * nocc;   // <= sig_rows
  if (!P->d_Sx) {
    GW_TRY(dalloc(P, &P->d_Sx, (size_t)rows_max));
    if (!P->fp64) {
      GW_TRY(dalloc(P, &P->d_Ux, (size_t)rows_max * P->Kx));
      GW_TRY(dalloc(P, &P->d_Vx32, (size_t)NN));
    }
  }
  const c128* evec = reinterpret_cast<const c128*>(P->p.evec);
  const c128* V = reinterpret_cast<const c128*>(P->p.V);
  GW_CUDA(cudaMemsetAsync(sigx, 0, sizeof(double) * P->NK * nsig, st));
  for (int q = 0; q < P->NK; ++q) {
    if (!P->fp64) launch_convert((int)NN, V + q * NN, P->d_Vx32, st);
    for (int kk0 = 0; kk0 < P->NK; kk0 += P->sig_nkk) {
      const int nkk = std::min(P->sig_nkk, P->NK - kk0);
      const int R = nkk * nsig * nocc;
      if (P->fp64) {
        c128* A = static_cast<c128*>(P->d_A);
        c128* U = static_cast<c128*>(P->d_U);
        launch_mgen<double>(P->geom, static_cast<const c128*>(P->d_T1), nullptr, evec, q, kk0, nkk,
                            MAP_K_IS_KK_MINUS_Q, P->p.sigma_lo, nsig, 0, nocc, A, N, 1, st);
        launch_zgemm<double>(R, N, N, c128{1, 0}, A, N, 0, OP_N, V + q * NN, N, 0, OP_N, c128{0, 0}, U, N, 0, 1, st);
        launch_rowdot<double>(R, N, U, A, N, nullptr, P->d_Sx, 0, 1, st);
      } else {
        c64* A = static_cast<c64*>(P->d_A);
        if (!P->mtune.run(0, nsig, nocc, st, [&](int v) {
              launch_mgen<float>(P->geom, static_cast<const c64*>(P->d_T1), nullptr, evec, q, kk0, nkk,
                                 MAP_K_IS_KK_MINUS_Q, P->p.sigma_lo, nsig, 0, nocc, A, P->Kx, 1, st, v);
            }))
          return fail(GW_ERR_CUDA, "M kernel autotuner: CUDA error");
        launch_zgemm<float>(R, N, N, c64{1, 0}, A, P->Kx, 0, OP_N, P->d_Vx32, N, 0, OP_N, c64{0, 0}, P->d_Ux, P->Kx,
                            0, 1, st);
        launch_rowdot<float>(R, N, P->d_Ux, A, P->Kx, nullptr, P->d_Sx, 0, 1, st);
      }
      ++g_launch_count, k_sigx_accum<<<(nkk * nsig + 127) / 128, 128, 0, st>>>(nkk, kk0, nsig, nocc, P->d_Sx,
                                                                             -1.0 / P->NK, sigx);
    }
    GW_TRY(check_launch(P, "gw_sigma_x"));
  }
  return GW_OK;
}

}  // extern "C"
