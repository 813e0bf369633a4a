// Learned frequency surrogate: the network f(x) = L x + s * MLP(x), its training (forward,
// backward, Adam, closed-form ridge fit of L) and inference. The paper has no counterpart;
// the model predicts the mode diagonal of eps~^-1 - 1 on the fine frequencies of the grid
// from its values on a coarse subset.
//
//   MLP(x) = W4 h3 + b4,  h3 = silu(W3 h2 + b3),  h2 = silu(W2 h1 + b2),  h1 = silu(W1 x + b1)
//
// Parameters: one fp32 vector, W1 [H][I], b1 [H], W2 [H][H], b2 [H], W3 [H][H], b3 [H],
// W4 [O][H], b4 [O], L [O][I], s [1] (row-major). Matrix products read bf16 copies of
// W1..W4 and accumulate in fp32; biases, L and s are used in fp32. Adam trains W1..b4;
// L and s come from gw_surrogate_fit_linear (ridge normal equations in FP64).
#include "gw_internal.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

using namespace gw;

namespace {

thread_local std::string g_mlp_err;

gw_status mfail(gw_status s, const std::string& m) {
  g_mlp_err = m;
  gw_set_last_error(m);
  return s;
}

#define MLP_CUDA(call)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return mfail(GW_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define MLP_TRY(x)               \
  do {                           \
    gw_status s_ = (x);          \
    if (s_ != GW_OK) return s_;  \
  } while (0)

struct Offs {
  long long W1, b1, W2, b2, W3, b3, W4, b4, L, s, P;
};

Offs offsets(int I, int H, int O) {
  Offs o{};
  long long p = 0;
  o.W1 = p; p += (long long)H * I;
  o.b1 = p; p += H;
  o.W2 = p; p += (long long)H * H;
  o.b2 = p; p += H;
  o.W3 = p; p += (long long)H * H;
  o.b3 = p; p += H;
  o.W4 = p; p += (long long)O * H;
  o.b4 = p; p += O;
  o.L = p; p += (long long)O * I;
  o.s = p; p += 1;
  o.P = p;
  return o;
}

// ---------------------------------------------------------------------------------------------
// C[M][N] = alpha * sum_k A(m,k) B(k,n) + beta * C + bias_scale * bias[n]
//   A(m,k) = tA ? A[k*lda + m] : A[m*lda + k]   (fp32)
//   B(k,n) = tB ? B[n*ldb + k] : B[k*ldb + n]   (fp32 or bf16, converted to fp32)
// 64x64 tiles, k-steps of 16, 256 threads with 4x4 outputs each (strided by 16).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename TB>
__global__ void __launch_bounds__(256) k_mm(int M, int N, int K, const float* __restrict__ A, int lda, int tA,
                                            const TB* __restrict__ B, int ldb, int tB, float* __restrict__ C, int ldc,
                                            float alpha, float beta, const float* __restrict__ bias,
                                            float bias_scale) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + 256 * r;
      int mm, kk;
      if (tA) { kk = e / 64; mm = e % 64; } else { mm = e / 16; kk = e % 16; }
      const int gm = m0 + mm, gk = k0 + kk;
      float va = 0.f;
      if (gm < M && gk < K) va = tA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
      As[kk][mm] = va;
      int nn, kb;
      if (tB) { nn = e / 16; kb = e % 16; } else { kb = e / 64; nn = e % 64; }
      const int gn = n0 + nn, gk2 = k0 + kb;
      float vb = 0.f;
      if (gn < N && gk2 < K) vb = tB ? to_f(B[(long long)gn * ldb + gk2]) : to_f(B[(long long)gk2 * ldb + gn]);
      Bs[kb][nn] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= N) continue;
      float v = alpha * acc[i][j];
      if (beta != 0.f) v += beta * C[(long long)m * ldc + n];
      if (bias) v += bias_scale * bias[n];
      C[(long long)m * ldc + n] = v;
    }
  }
}

template <typename TB>
void mm(int M, int N, int K, const float* A, int lda, int tA, const TB* B, int ldb, int tB, float* C, int ldc,
        float alpha, float beta, const float* bias, float bias_scale, cudaStream_t st) {
  if (M <= 0 || N <= 0) return;
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  ++g_launch_count, k_mm<TB><<<grid, 256, 0, st>>>(M, N, K, A, lda, tA, B, ldb, tB, C, ldc, alpha, beta, bias,
                                                   bias_scale);
}

// ---------------------------------------------------------------------------------------------
// elementwise pieces
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float sigm(float z) { return 1.f / (1.f + expf(-z)); }

__global__ void k_silu_fwd(long long n, const float* __restrict__ Z, float* __restrict__ Hh) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float z = Z[i];
    Hh[i] = z * sigm(z);
  }
}

// dZ = dH * silu'(Z), silu'(z) = s (1 + z (1 - s)), s = sigmoid(z)
__global__ void k_silu_bwd(long long n, const float* __restrict__ dH, const float* __restrict__ Z,
                           float* __restrict__ dZ) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float z = Z[i], s = sigm(z);
    dZ[i] = dH[i] * s * (1.f + z * (1.f - s));
  }
}

// out[n] = alpha * sum_m A[m][n]  (one thread per column, rows in order)
__global__ void k_colsum(int M, int N, const float* __restrict__ A, float alpha, float* __restrict__ out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float acc = 0.f;
  for (int m = 0; m < M; ++m) acc += A[(long long)m * N + n];
  out[n] = alpha * acc;
}

// F = F + s G (F holds x L^T on entry); R = F - Y; dF = 2 R / (B n_out); loss += sum R^2 / (B n_out)
__global__ void k_mse(long long n, float inv, float s, float* __restrict__ F, const float* __restrict__ G,
                      const float* __restrict__ Y, float* __restrict__ dF, double* __restrict__ loss) {
  __shared__ double red[256];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float f = F[i] + s * G[i];
    F[i] = f;
    if (!Y) continue;
    const float r = f - Y[i];
    if (dF) dF[i] = 2.f * r * inv;
    acc += (double)r * r;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss) atomicAdd(loss, red[0] * (double)inv);
}

// bf16 copies of the weight matrices (round to nearest even); other entries copied too
__global__ void k_to_bf16(long long n, const float* __restrict__ a, __nv_bfloat16* __restrict__ b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16_rn(a[i]);
}

// Adam (Kingma & Ba, Algorithm 1) on theta[0 .. n), step t = *t_dev + 1; refreshes the bf16 copy
__global__ void k_adam(long long n, float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ wb, const int* __restrict__ t_dev, float lr,
                       float b1, float b2, float eps) {
  const int t = *t_dev + 1;
  const float c1 = 1.f / (1.f - powf(b1, (float)t)), c2 = 1.f / (1.f - powf(b2, (float)t));
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float w = th[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    th[i] = w;
    wb[i] = __float2bfloat16_rn(w);
  }
}

// rows of the next batch: xb[i] = x[perm[step * B + i]], yb likewise
__global__ void k_gather(int B, int I, int O, const float* __restrict__ x, const float* __restrict__ y,
                         const int* __restrict__ perm, const int* __restrict__ step, float* __restrict__ xb,
                         float* __restrict__ yb) {
  const int i = blockIdx.x;
  const int r = perm[(long long)(*step) * B + i];
  for (int j = threadIdx.x; j < I; j += blockDim.x) xb[(long long)i * I + j] = x[(long long)r * I + j];
  for (int j = threadIdx.x; j < O; j += blockDim.x) yb[(long long)i * O + j] = y[(long long)r * O + j];
}

__global__ void k_tick(int* __restrict__ step, int* __restrict__ t) {
  ++*step;
  ++*t;
}

// FP64 normal equations of the ridge fit: G += x^T x, R += x^T y over a chunk of rows per block
__global__ void k_gram(long long n, int I, int O, const float* __restrict__ x, const float* __restrict__ y,
                       long long rows_per_block, double* __restrict__ G, double* __restrict__ R) {
  const long long r0 = blockIdx.x * rows_per_block, r1 = min(n, r0 + rows_per_block);
  const int outs = I * (I + O);
  for (int e = threadIdx.x; e < outs; e += blockDim.x) {
    const int i = e / (I + O), j = e % (I + O);
    double acc = 0.0;
    if (j < I) {
      for (long long r = r0; r < r1; ++r) acc += (double)x[r * I + i] * (double)x[r * I + j];
      atomicAdd(&G[i * I + j], acc);
    } else {
      const int o = j - I;
      for (long long r = r0; r < r1; ++r) acc += (double)x[r * I + i] * (double)y[r * O + o];
      atomicAdd(&R[i * O + o], acc);
    }
  }
}

// (G + lam 1) L^T = R by Cholesky in shared memory (I <= 64); writes L [O][I] (fp32) into theta.
// One block; status bit ST_NOT_PD if a pivot is not positive.
__global__ void k_ridge_solve(int I, int O, const double* __restrict__ G, const double* __restrict__ R, double lam,
                              float* __restrict__ Lout, int* __restrict__ status) {
  __shared__ double c[64][65];
  for (int e = threadIdx.x; e < I * I; e += blockDim.x) c[e / I][e % I] = G[e] + (e / I == e % I ? lam : 0.0);
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int j = 0; j < I; ++j) {
      double d = c[j][j];
      for (int k = 0; k < j; ++k) d -= c[j][k] * c[j][k];
      if (!(d > 0.0)) {
        atomicOr(status, ST_NOT_PD);
        d = 1e-300;
      }
      c[j][j] = sqrt(d);
      for (int i = j + 1; i < I; ++i) {
        double s = c[i][j];
        for (int k = 0; k < j; ++k) s -= c[i][k] * c[j][k];
        c[i][j] = s / c[j][j];
      }
    }
  }
  __syncthreads();
  for (int o = threadIdx.x; o < O; o += blockDim.x) {
    double z[64];
    for (int i = 0; i < I; ++i) {  // forward: C z = r
      double s = R[i * O + o];
      for (int k = 0; k < i; ++k) s -= c[i][k] * z[k];
      z[i] = s / c[i][i];
    }
    for (int i = I - 1; i >= 0; --i) {  // backward: C^T l = z
      double s = z[i];
      for (int k = i + 1; k < I; ++k) s -= c[k][i] * z[k];
      z[i] = s / c[i][i];
    }
    for (int i = 0; i < I; ++i) Lout[(long long)o * I + i] = (float)z[i];
  }
}

// sum of squared residuals of the linear map in FP64: sum (y - x L^T)^2
__global__ void k_lin_resid(long long n, int I, int O, const float* __restrict__ x, const float* __restrict__ y,
                            const float* __restrict__ L, double* __restrict__ out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * O;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / O;
    const int o = (int)(e % O);
    double f = 0.0;
    for (int i = 0; i < I; ++i) f += (double)L[(long long)o * I + i] * (double)x[r * I + i];
    const double d = (double)y[e] - f;
    acc += d * d;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, red[0]);
}

inline int ew_grid(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 16); }

}  // namespace

namespace {
// residual targets of the MLP in FP64: yr = (y - x L^T) / s
__global__ void k_resid_targets(long long n, int I, int O, const float* __restrict__ x, const float* __restrict__ y,
                                const float* __restrict__ L, const float* __restrict__ s_dev, float* __restrict__ yr) {
  const double inv_s = 1.0 / (double)(*s_dev);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * O;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / O;
    const int o = (int)(e % O);
    double f = 0.0;
    for (int i = 0; i < I; ++i) f += (double)L[(long long)o * I + i] * (double)x[r * I + i];
    yr[e] = (float)(((double)y[e] - f) * inv_s);
  }
}

// loss += sum (G - Y)^2 / (B O) and dG = 2 (G - Y) / (B O)   (residual form, no linear part)
__global__ void k_mse_res(long long n, float inv, const float* __restrict__ G, const float* __restrict__ Y,
                          float* __restrict__ dG, double* __restrict__ loss) {
  __shared__ double red[256];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float r = G[i] - Y[i];
    dG[i] = 2.f * r * inv;
    acc += (double)r * r;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] * (double)inv);
}
}  // namespace

// ---------------------------------------------------------------------------------------------
// the model
// ---------------------------------------------------------------------------------------------
struct gw_surrogate_s {
  int I = 0, H = 0, O = 0;
  Offs off{};
  cudaStream_t st = nullptr;     // the model's own stream (non-blocking)
  cudaStream_t user = nullptr;   // the caller's stream, ordered against st by events
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  float* th = nullptr;           // fp32 parameters [P]
  __nv_bfloat16* wb = nullptr;   // bf16 copy [P] (matrix entries are the ones used)
  float* grad = nullptr;         // [P]
  float *am = nullptr, *av = nullptr;  // Adam moments [P]
  int* d_ctr = nullptr;          // [0] batch index within the epoch, [1] Adam step count
  double* d_acc = nullptr;       // [0] loss accumulator, [1..] scratch
  int* d_status = nullptr;
  float h_s = 1.f;               // host copy of the output scale s
  // activations for up to cap rows
  int cap = 0;
  float *xb = nullptr, *yb = nullptr, *Z1 = nullptr, *H1 = nullptr, *Z2 = nullptr, *H2 = nullptr, *Z3 = nullptr,
        *H3 = nullptr, *G = nullptr, *F = nullptr, *dG = nullptr, *dA = nullptr, *dB = nullptr;
  std::vector<void*> allocs;
};

namespace {

gw_status salloc(gw_surrogate_s* m, void** p, size_t bytes) {
  ++::gw::g_alloc_count;
  cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return mfail(GW_ERR_NOMEM, "surrogate: cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  m->allocs.push_back(*p);
  return GW_OK;
}

template <typename T>
gw_status salloc_n(gw_surrogate_s* m, T** p, size_t n) {
  return salloc(m, reinterpret_cast<void**>(p), n * sizeof(T));
}

void sfree(gw_surrogate_s* m, void* p) {
  if (!p) return;
  cudaFree(p);
  auto it = std::find(m->allocs.begin(), m->allocs.end(), p);
  if (it != m->allocs.end()) m->allocs.erase(it);
}

gw_status ensure_cap(gw_surrogate_s* m, int rows) {
  if (rows <= m->cap) return GW_OK;
  float** bufs[] = {&m->xb, &m->yb, &m->Z1, &m->H1, &m->Z2, &m->H2, &m->Z3, &m->H3, &m->G, &m->F, &m->dG, &m->dA, &m->dB};
  for (float** b : bufs) {
    sfree(m, *b);
    *b = nullptr;
  }
  const size_t r = (size_t)rows;
  const size_t wI = m->I, wH = m->H, wO = m->O;
  MLP_TRY(salloc_n(m, &m->xb, r * wI));
  MLP_TRY(salloc_n(m, &m->yb, r * wO));
  MLP_TRY(salloc_n(m, &m->Z1, r * wH));
  MLP_TRY(salloc_n(m, &m->H1, r * wH));
  MLP_TRY(salloc_n(m, &m->Z2, r * wH));
  MLP_TRY(salloc_n(m, &m->H2, r * wH));
  MLP_TRY(salloc_n(m, &m->Z3, r * wH));
  MLP_TRY(salloc_n(m, &m->H3, r * wH));
  MLP_TRY(salloc_n(m, &m->G, r * wO));
  MLP_TRY(salloc_n(m, &m->F, r * wO));
  MLP_TRY(salloc_n(m, &m->dG, r * wO));
  MLP_TRY(salloc_n(m, &m->dA, r * wH));
  MLP_TRY(salloc_n(m, &m->dB, r * wH));
  m->cap = rows;
  return GW_OK;
}

// G = MLP(x) (without the output scale s) for B rows of x; activations kept for backward
void forward_mlp(gw_surrogate_s* m, const float* x, int B, float* G, cudaStream_t st) {
  const int I = m->I, H = m->H, O = m->O;
  const Offs& o = m->off;
  const long long nh = (long long)B * H;
  mm<__nv_bfloat16>(B, H, I, x, I, 0, m->wb + o.W1, I, 1, m->Z1, H, 1.f, 0.f, m->th + o.b1, 1.f, st);
  ++g_launch_count, k_silu_fwd<<<ew_grid(nh), 256, 0, st>>>(nh, m->Z1, m->H1);
  mm<__nv_bfloat16>(B, H, H, m->H1, H, 0, m->wb + o.W2, H, 1, m->Z2, H, 1.f, 0.f, m->th + o.b2, 1.f, st);
  ++g_launch_count, k_silu_fwd<<<ew_grid(nh), 256, 0, st>>>(nh, m->Z2, m->H2);
  mm<__nv_bfloat16>(B, H, H, m->H2, H, 0, m->wb + o.W3, H, 1, m->Z3, H, 1.f, 0.f, m->th + o.b3, 1.f, st);
  ++g_launch_count, k_silu_fwd<<<ew_grid(nh), 256, 0, st>>>(nh, m->Z3, m->H3);
  mm<__nv_bfloat16>(B, O, H, m->H3, H, 0, m->wb + o.W4, H, 1, G, O, 1.f, 0.f, m->th + o.b4, 1.f, st);
}

// gradients of the W/b parameters from dG = dLoss/d(MLP output) for the B rows of x (alpha
// scales every gradient, e.g. by s); fills m->grad[W1 .. b4]
void backward_mlp(gw_surrogate_s* m, const float* x, int B, const float* dG, float alpha, cudaStream_t st) {
  const int I = m->I, H = m->H, O = m->O;
  const Offs& o = m->off;
  const long long nh = (long long)B * H;
  float* g = m->grad;
  mm<float>(O, H, B, dG, O, 1, m->H3, H, 0, g + o.W4, H, alpha, 0.f, nullptr, 0.f, st);
  ++g_launch_count, k_colsum<<<(O + 127) / 128, 128, 0, st>>>(B, O, dG, alpha, g + o.b4);
  mm<__nv_bfloat16>(B, H, O, dG, O, 0, m->wb + o.W4, H, 0, m->dA, H, alpha, 0.f, nullptr, 0.f, st);
  ++g_launch_count, k_silu_bwd<<<ew_grid(nh), 256, 0, st>>>(nh, m->dA, m->Z3, m->dB);  // dZ3
  mm<float>(H, H, B, m->dB, H, 1, m->H2, H, 0, g + o.W3, H, 1.f, 0.f, nullptr, 0.f, st);
  ++g_launch_count, k_colsum<<<(H + 127) / 128, 128, 0, st>>>(B, H, m->dB, 1.f, g + o.b3);
  mm<__nv_bfloat16>(B, H, H, m->dB, H, 0, m->wb + o.W3, H, 0, m->dA, H, 1.f, 0.f, nullptr, 0.f, st);
  ++g_launch_count, k_silu_bwd<<<ew_grid(nh), 256, 0, st>>>(nh, m->dA, m->Z2, m->dB);  // dZ2
  mm<float>(H, H, B, m->dB, H, 1, m->H1, H, 0, g + o.W2, H, 1.f, 0.f, nullptr, 0.f, st);
  ++g_launch_count, k_colsum<<<(H + 127) / 128, 128, 0, st>>>(B, H, m->dB, 1.f, g + o.b2);
  mm<__nv_bfloat16>(B, H, H, m->dB, H, 0, m->wb + o.W2, H, 0, m->dA, H, 1.f, 0.f, nullptr, 0.f, st);
  ++g_launch_count, k_silu_bwd<<<ew_grid(nh), 256, 0, st>>>(nh, m->dA, m->Z1, m->dB);  // dZ1
  mm<float>(H, I, B, m->dB, H, 1, x, I, 0, g + o.W1, I, 1.f, 0.f, nullptr, 0.f, st);
  ++g_launch_count, k_colsum<<<(H + 127) / 128, 128, 0, st>>>(B, H, m->dB, 1.f, g + o.b1);
}

gw_status begin(gw_surrogate_s* m) {
  MLP_CUDA(cudaEventRecord(m->ev_in, m->user));
  MLP_CUDA(cudaStreamWaitEvent(m->st, m->ev_in, 0));
  return GW_OK;
}

gw_status finish(gw_surrogate_s* m, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return mfail(GW_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  MLP_CUDA(cudaEventRecord(m->ev_out, m->st));
  MLP_CUDA(cudaStreamWaitEvent(m->user, m->ev_out, 0));
  return GW_OK;
}

}  // namespace

namespace {

__global__ void k_scale_copy(long long n, float s, const float* __restrict__ a, float* __restrict__ b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = s * a[i];
}

uint64_t splitmix64(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

bool dims_ok(const gw_surrogate_dims* d) {
  return d && d->n_in >= 1 && d->n_in <= 64 && d->n_hidden >= 1 && d->n_hidden <= 4096 && d->n_out >= 1 &&
         d->n_out <= 1024;
}

constexpr int kChunk = 8192;  // rows per forward pass of gw_surrogate_forward

}  // namespace

namespace gw {

// g = s * MLP(x) for n <= 4096 rows on stream st (used by the plan's surrogate pass)
gw_status sur_correction(gw_surrogate_s* m, const float* x, int n, float* g_out, cudaStream_t st) {
  if (n > 4096) return mfail(GW_ERR_ARG, "surrogate: too many modes for one pass");
  MLP_TRY(ensure_cap(m, std::max(n, 1)));
  forward_mlp(m, x, n, m->G, st);
  const long long no = (long long)n * m->O;
  ++g_launch_count, k_scale_copy<<<ew_grid(no), 256, 0, st>>>(no, m->h_s, m->G, g_out);
  return GW_OK;
}

int sur_n_in(const gw_surrogate_s* m) { return m->I; }
int sur_n_out(const gw_surrogate_s* m) { return m->O; }
const float* sur_linear(const gw_surrogate_s* m) { return m->th + m->off.L; }

}  // namespace gw

extern "C" {

gw_status gw_surrogate_param_count(const gw_surrogate_dims* dims, int64_t* count) {
  if (!dims_ok(dims) || !count) return mfail(GW_ERR_ARG, "surrogate: bad dims or NULL count");
  *count = offsets(dims->n_in, dims->n_hidden, dims->n_out).P;
  return GW_OK;
}

gw_status gw_surrogate_create(const gw_surrogate_dims* dims, const float* params, void* stream, gw_surrogate* out) {
  if (!out) return mfail(GW_ERR_ARG, "surrogate: out is NULL");
  *out = nullptr;
  if (!dims_ok(dims)) return mfail(GW_ERR_ARG, "surrogate: dims out of range (n_in 1..64, n_hidden 1..4096, n_out 1..1024)");
  if (!params) return mfail(GW_ERR_ARG, "surrogate: params is NULL");
  auto* m = new (std::nothrow) gw_surrogate_s();
  if (!m) return mfail(GW_ERR_NOMEM, "surrogate: host allocation failed");
  m->I = dims->n_in;
  m->H = dims->n_hidden;
  m->O = dims->n_out;
  m->off = offsets(m->I, m->H, m->O);
  m->user = static_cast<cudaStream_t>(stream);
  auto fail_destroy = [&](gw_status s) {
    gw_surrogate_destroy(m);
    return s;
  };
  if (cudaStreamCreateWithFlags(&m->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&m->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&m->ev_out, cudaEventDisableTiming) != cudaSuccess)
    return fail_destroy(mfail(GW_ERR_CUDA, "surrogate: stream/event creation failed"));
  const size_t P = (size_t)m->off.P;
  gw_status s;
  if ((s = salloc_n(m, &m->th, P)) != GW_OK || (s = salloc_n(m, &m->wb, P)) != GW_OK ||
      (s = salloc_n(m, &m->grad, P)) != GW_OK || (s = salloc_n(m, &m->am, P)) != GW_OK ||
      (s = salloc_n(m, &m->av, P)) != GW_OK || (s = salloc_n(m, &m->d_ctr, 4)) != GW_OK ||
      (s = salloc_n(m, &m->d_acc, 2 + (size_t)m->I * (m->I + m->O))) != GW_OK ||
      (s = salloc_n(m, &m->d_status, 1)) != GW_OK)
    return fail_destroy(s);
  if ((s = begin(m)) != GW_OK) return fail_destroy(s);
  cudaMemcpyAsync(m->th, params, P * sizeof(float), cudaMemcpyDeviceToDevice, m->st);
  cudaMemsetAsync(m->am, 0, P * sizeof(float), m->st);
  cudaMemsetAsync(m->av, 0, P * sizeof(float), m->st);
  cudaMemsetAsync(m->grad, 0, P * sizeof(float), m->st);
  cudaMemsetAsync(m->d_ctr, 0, 4 * sizeof(int), m->st);
  ++g_launch_count, k_to_bf16<<<ew_grid((long long)P), 256, 0, m->st>>>((long long)P, m->th, m->wb);
  float hs = 1.f;
  cudaMemcpyAsync(&hs, m->th + m->off.s, sizeof(float), cudaMemcpyDeviceToHost, m->st);
  if (cudaStreamSynchronize(m->st) != cudaSuccess) return fail_destroy(mfail(GW_ERR_CUDA, "surrogate: create failed"));
  m->h_s = hs;
  if ((s = finish(m, "gw_surrogate_create")) != GW_OK) return fail_destroy(s);
  *out = m;
  return GW_OK;
}

gw_status gw_surrogate_destroy(gw_surrogate m) {
  if (!m) return GW_OK;
  if (m->st) cudaStreamSynchronize(m->st);
  for (void* p : m->allocs) cudaFree(p);
  if (m->ev_in) cudaEventDestroy(m->ev_in);
  if (m->ev_out) cudaEventDestroy(m->ev_out);
  if (m->st) cudaStreamDestroy(m->st);
  delete m;
  return GW_OK;
}

gw_status gw_surrogate_get_params(gw_surrogate m, float* params) {
  if (!m || !params) return mfail(GW_ERR_ARG, "surrogate: NULL argument");
  MLP_TRY(begin(m));
  MLP_CUDA(cudaMemcpyAsync(params, m->th, (size_t)m->off.P * sizeof(float), cudaMemcpyDeviceToDevice, m->st));
  return finish(m, "gw_surrogate_get_params");
}

gw_status gw_surrogate_set_params(gw_surrogate m, const float* params) {
  if (!m || !params) return mfail(GW_ERR_ARG, "surrogate: NULL argument");
  MLP_TRY(begin(m));
  const long long P = m->off.P;
  MLP_CUDA(cudaMemcpyAsync(m->th, params, (size_t)P * sizeof(float), cudaMemcpyDeviceToDevice, m->st));
  ++g_launch_count, k_to_bf16<<<ew_grid(P), 256, 0, m->st>>>(P, m->th, m->wb);
  float hs = 1.f;
  MLP_CUDA(cudaMemcpyAsync(&hs, m->th + m->off.s, sizeof(float), cudaMemcpyDeviceToHost, m->st));
  MLP_CUDA(cudaStreamSynchronize(m->st));
  m->h_s = hs;
  return finish(m, "gw_surrogate_set_params");
}

gw_status gw_surrogate_forward(gw_surrogate m, const float* x, int64_t n, float* f, float* g) {
  if (!m || !x || (!f && !g) || n < 0) return mfail(GW_ERR_ARG, "surrogate: bad forward arguments");
  MLP_TRY(begin(m));
  const int I = m->I, O = m->O;
  MLP_TRY(ensure_cap(m, (int)std::min<int64_t>(std::max<int64_t>(n, 1), kChunk)));
  for (int64_t r0 = 0; r0 < n; r0 += kChunk) {
    const int B = (int)std::min<int64_t>(kChunk, n - r0);
    const float* xr = x + r0 * I;
    forward_mlp(m, xr, B, m->G, m->st);
    const long long no = (long long)B * O;
    if (g) ++g_launch_count, k_scale_copy<<<ew_grid(no), 256, 0, m->st>>>(no, m->h_s, m->G, g + r0 * O);
    if (f) {
      float* fr = f + r0 * O;
      mm<float>(B, O, I, xr, I, 0, m->th + m->off.L, I, 1, fr, O, 1.f, 0.f, nullptr, 0.f, m->st);
      ++g_launch_count, k_mse<<<ew_grid(no), 256, 0, m->st>>>(no, 0.f, m->h_s, fr, m->G, nullptr, nullptr, nullptr);
    }
  }
  return finish(m, "gw_surrogate_forward");
}

gw_status gw_surrogate_loss_grad(gw_surrogate m, const float* x, const float* y, int64_t n, double* loss,
                                 float* grad) {
  if (!m || !x || !y || !loss || !grad || n < 1 || n > 65536)
    return mfail(GW_ERR_ARG, "surrogate: bad loss_grad arguments (1 <= n <= 65536)");
  MLP_TRY(begin(m));
  const int I = m->I, O = m->O, B = (int)n;
  const Offs& o = m->off;
  MLP_TRY(ensure_cap(m, B));
  MLP_CUDA(cudaMemsetAsync(m->d_acc, 0, sizeof(double), m->st));
  forward_mlp(m, x, B, m->G, m->st);
  mm<float>(B, O, I, x, I, 0, m->th + o.L, I, 1, m->F, O, 1.f, 0.f, nullptr, 0.f, m->st);
  const long long no = (long long)B * O;
  ++g_launch_count, k_mse<<<ew_grid(no), 256, 0, m->st>>>(no, 1.f / (float)no, m->h_s, m->F, m->G, y, m->dG,
                                                          m->d_acc);
  backward_mlp(m, x, B, m->dG, m->h_s, m->st);
  mm<float>(O, I, B, m->dG, O, 1, x, I, 0, m->grad + o.L, I, 1.f, 0.f, nullptr, 0.f, m->st);
  MLP_CUDA(cudaMemsetAsync(m->grad + o.s, 0, sizeof(float), m->st));
  MLP_CUDA(cudaMemcpyAsync(grad, m->grad, (size_t)o.P * sizeof(float), cudaMemcpyDeviceToDevice, m->st));
  double h = 0.0;
  MLP_CUDA(cudaMemcpyAsync(&h, m->d_acc, sizeof(double), cudaMemcpyDeviceToHost, m->st));
  MLP_CUDA(cudaStreamSynchronize(m->st));
  *loss = h;
  return finish(m, "gw_surrogate_loss_grad");
}

gw_status gw_surrogate_fit_linear(gw_surrogate m, const float* x, const float* y, int64_t n, double ridge,
                                  double* rms) {
  if (!m || !x || !y || n < 1 || !(ridge >= 0.0)) return mfail(GW_ERR_ARG, "surrogate: bad fit_linear arguments");
  MLP_TRY(begin(m));
  const int I = m->I, O = m->O;
  double* G = m->d_acc + 2;
  double* R = G + (size_t)I * I;
  MLP_CUDA(cudaMemsetAsync(m->d_acc, 0, (2 + (size_t)I * (I + O)) * sizeof(double), m->st));
  MLP_CUDA(cudaMemsetAsync(m->d_status, 0, sizeof(int), m->st));
  const long long rpb = std::max<long long>(256, (n + 152 * 4 - 1) / (152 * 4));
  const int nblk = (int)((n + rpb - 1) / rpb);
  ++g_launch_count, k_gram<<<nblk, 256, 0, m->st>>>(n, I, O, x, y, rpb, G, R);
  ++g_launch_count, k_ridge_solve<<<1, 64, 0, m->st>>>(I, O, G, R, ridge * (double)n, m->th + m->off.L, m->d_status);
  ++g_launch_count, k_lin_resid<<<ew_grid(n * O), 256, 0, m->st>>>(n, I, O, x, y, m->th + m->off.L, m->d_acc);
  double ss = 0.0;
  int stt = 0;
  MLP_CUDA(cudaMemcpyAsync(&ss, m->d_acc, sizeof(double), cudaMemcpyDeviceToHost, m->st));
  MLP_CUDA(cudaMemcpyAsync(&stt, m->d_status, sizeof(int), cudaMemcpyDeviceToHost, m->st));
  MLP_CUDA(cudaStreamSynchronize(m->st));
  if (stt & ST_NOT_PD) return mfail(GW_ERR_NOT_PD, "surrogate: x^T x + ridge is not positive definite");
  const double r = std::sqrt(ss / ((double)n * O));
  const float s = (r > 0.0 && std::isfinite(r)) ? (float)r : 1.f;
  MLP_CUDA(cudaMemcpyAsync(m->th + m->off.s, &s, sizeof(float), cudaMemcpyHostToDevice, m->st));
  MLP_CUDA(cudaStreamSynchronize(m->st));
  m->h_s = s;
  if (rms) *rms = r;
  return finish(m, "gw_surrogate_fit_linear");
}

gw_status gw_surrogate_fit_moments(gw_surrogate m, const double* moments, double ridge) {
  if (!m || !moments || !(ridge >= 0.0)) return mfail(GW_ERR_ARG, "surrogate: bad fit_moments arguments");
  MLP_TRY(begin(m));
  const int I = m->I, O = m->O;
  double* G = m->d_acc + 2;
  double* R = G + (size_t)I * I;
  std::vector<double> h((size_t)I * (I + O));
  MLP_CUDA(cudaMemcpyAsync(h.data(), moments, h.size() * sizeof(double), cudaMemcpyDeviceToHost, m->st));
  MLP_CUDA(cudaMemcpy2DAsync(G, I * sizeof(double), moments, (I + O) * sizeof(double), I * sizeof(double), I,
                             cudaMemcpyDeviceToDevice, m->st));
  MLP_CUDA(cudaMemcpy2DAsync(R, O * sizeof(double), moments + I, (I + O) * sizeof(double), O * sizeof(double), I,
                             cudaMemcpyDeviceToDevice, m->st));
  MLP_CUDA(cudaMemsetAsync(m->d_status, 0, sizeof(int), m->st));
  MLP_CUDA(cudaStreamSynchronize(m->st));
  double tr = 0.0;
  for (int i = 0; i < I; ++i) tr += h[(size_t)i * (I + O) + i];
  ++g_launch_count, k_ridge_solve<<<1, 64, 0, m->st>>>(I, O, G, R, ridge * tr / I, m->th + m->off.L, m->d_status);
  int stt = 0;
  MLP_CUDA(cudaMemcpyAsync(&stt, m->d_status, sizeof(int), cudaMemcpyDeviceToHost, m->st));
  MLP_CUDA(cudaStreamSynchronize(m->st));
  if (stt & ST_NOT_PD) return mfail(GW_ERR_NOT_PD, "surrogate: the coarse moment matrix + ridge is not positive definite");
  return finish(m, "gw_surrogate_fit_moments");
}

gw_status gw_surrogate_fit_scale(gw_surrogate m, const float* x, const float* y, int64_t n, double* rms) {
  if (!m || !x || !y || n < 1) return mfail(GW_ERR_ARG, "surrogate: bad fit_scale arguments");
  MLP_TRY(begin(m));
  const int I = m->I, O = m->O;
  MLP_CUDA(cudaMemsetAsync(m->d_acc, 0, sizeof(double), m->st));
  ++g_launch_count, k_lin_resid<<<ew_grid(n * O), 256, 0, m->st>>>(n, I, O, x, y, m->th + m->off.L, m->d_acc);
  double ss = 0.0;
  MLP_CUDA(cudaMemcpyAsync(&ss, m->d_acc, sizeof(double), cudaMemcpyDeviceToHost, m->st));
  MLP_CUDA(cudaStreamSynchronize(m->st));
  const double r = std::sqrt(ss / ((double)n * O));
  const float sc = (r > 0.0 && std::isfinite(r)) ? (float)r : 1.f;
  MLP_CUDA(cudaMemcpyAsync(m->th + m->off.s, &sc, sizeof(float), cudaMemcpyHostToDevice, m->st));
  MLP_CUDA(cudaStreamSynchronize(m->st));
  m->h_s = sc;
  if (rms) *rms = r;
  return finish(m, "gw_surrogate_fit_scale");
}

gw_status gw_surrogate_train(gw_surrogate m, const float* x, const float* y, int64_t n, int32_t epochs, int32_t batch,
                             double lr, uint64_t seed, double* loss_hist) {
  if (!m || !x || !y || n < 1 || n > (int64_t)1 << 30 || epochs < 0 || batch < 1 || batch > 4096 || batch > n ||
      !(lr > 0.0))
    return mfail(GW_ERR_ARG, "surrogate: bad train arguments (1 <= batch <= min(n, 4096), lr > 0)");
  MLP_TRY(begin(m));
  const int I = m->I, O = m->O, B = batch;
  const int nb = (int)(n / B);  // the last n % batch rows of each shuffled epoch are skipped
  MLP_TRY(ensure_cap(m, B));
  float* yr = nullptr;
  int* perm = nullptr;
  MLP_TRY(salloc_n(m, &yr, (size_t)n * O));
  gw_status st = salloc_n(m, &perm, (size_t)n);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  auto cleanup = [&](gw_status s) {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamSynchronize(m->st);
    sfree(m, yr);
    sfree(m, perm);
    return s;
  };
  if (st != GW_OK) return cleanup(st);
  // residual targets of the MLP: yr = (y - x L^T) / s, in FP64
  ++g_launch_count, k_resid_targets<<<ew_grid(n * O), 256, 0, m->st>>>(n, I, O, x, y, m->th + m->off.L,
                                                                       m->th + m->off.s, yr);
  // one training step (gather, forward, loss, backward, Adam, counters) as a CUDA graph
  const unsigned long long c0 = g_launch_count;
  if (cudaStreamBeginCapture(m->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return cleanup(mfail(GW_ERR_CUDA, "surrogate: stream capture failed to begin"));
  const long long no = (long long)B * O;
  ++g_launch_count, k_gather<<<B, 64, 0, m->st>>>(B, I, O, x, yr, perm, m->d_ctr, m->xb, m->yb);
  forward_mlp(m, m->xb, B, m->G, m->st);
  ++g_launch_count, k_mse_res<<<ew_grid(no), 256, 0, m->st>>>(no, 1.f / (float)no, m->G, m->yb, m->dG, m->d_acc);
  backward_mlp(m, m->xb, B, m->dG, 1.f, m->st);
  ++g_launch_count, k_adam<<<ew_grid(m->off.L), 256, 0, m->st>>>(m->off.L, m->th, m->grad, m->am, m->av, m->wb,
                                                                 m->d_ctr + 1, (float)lr, 0.9f, 0.999f, 1e-8f);
  ++g_launch_count, k_tick<<<1, 1, 0, m->st>>>(m->d_ctr, m->d_ctr + 1);
  cudaError_t ce = cudaStreamEndCapture(m->st, &graph);
  const unsigned long long per_step = g_launch_count - c0;
  g_launch_count = c0;
  if (ce != cudaSuccess || !graph) return cleanup(mfail(GW_ERR_CUDA, std::string("surrogate: capture: ") + cudaGetErrorString(ce)));
  if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
    return cleanup(mfail(GW_ERR_CUDA, "surrogate: graph instantiation failed"));
  std::vector<int> hp((size_t)n);
  uint64_t state = seed;
  const double s2 = (double)m->h_s * m->h_s;
  for (int e = 0; e < epochs; ++e) {
    for (int64_t i = 0; i < n; ++i) hp[i] = (int)i;
    for (int64_t i = n - 1; i > 0; --i) {  // Fisher-Yates with splitmix64
      const int64_t j = (int64_t)(splitmix64(state) % (uint64_t)(i + 1));
      std::swap(hp[i], hp[j]);
    }
    if (cudaMemcpyAsync(perm, hp.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice, m->st) != cudaSuccess ||
        cudaMemsetAsync(m->d_ctr, 0, sizeof(int), m->st) != cudaSuccess ||
        cudaMemsetAsync(m->d_acc, 0, sizeof(double), m->st) != cudaSuccess)
      return cleanup(mfail(GW_ERR_CUDA, "surrogate: epoch set-up failed"));
    for (int b = 0; b < nb; ++b) {
      if (cudaGraphLaunch(exec, m->st) != cudaSuccess) return cleanup(mfail(GW_ERR_CUDA, "surrogate: graph launch failed"));
    }
    g_launch_count += per_step * (unsigned long long)nb;
    double acc = 0.0;
    if (cudaMemcpyAsync(&acc, m->d_acc, sizeof(double), cudaMemcpyDeviceToHost, m->st) != cudaSuccess ||
        cudaStreamSynchronize(m->st) != cudaSuccess)
      return cleanup(mfail(GW_ERR_CUDA, "surrogate: training step failed"));
    if (loss_hist) loss_hist[e] = s2 * acc / std::max(nb, 1);
  }
  gw_status fs = finish(m, "gw_surrogate_train");
  return cleanup(fs);
}

}  // extern "C"
