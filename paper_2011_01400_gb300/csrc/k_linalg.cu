// CUDA-core linear algebra of the G0W0 path: the generic complex GEMM used by the
// FP64 method and by the V^1/2 Newton-Schulz iteration, the FP64 chi0 contraction,
// the FP64 Cholesky factorisation + inversion of eps~, and the q = 0 helpers.
#include "gw_internal.h"

namespace gw {

// ---------------------------------------------------------------------------------------------
// Generic batched complex GEMM, C = alpha op(A) op(B) + beta C. 64x64 tile, 256 threads,
// 4x4 outputs per thread, K chunk 8.
// ---------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ cplx<T> load_op(const cplx<T>* X, long long ld, int r, int c, int op) {
  // element (r, c) of op(X)
  cplx<T> v = (op == OP_N || op == OP_CONJ) ? X[(long long)r * ld + c] : X[(long long)c * ld + r];
  if (op == OP_C || op == OP_CONJ) v.im = -v.im;
  return v;
}

template <typename T>
__global__ void __launch_bounds__(256) k_zgemm(int m, int n, int k, cplx<T> alpha, const cplx<T>* __restrict__ A,
                                               long long lda, long long sA, int opA, const cplx<T>* __restrict__ B,
                                               long long ldb, long long sB, int opB, cplx<T> beta,
                                               cplx<T>* __restrict__ C, long long ldc, long long sC) {
  __shared__ cplx<T> As[8][64 + 1];
  __shared__ cplx<T> Bs[8][64 + 1];
  const int bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  cplx<T> acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = {0, 0};
  for (int k0 = 0; k0 < k; k0 += 8) {
    for (int e = threadIdx.x; e < 8 * 64; e += 256) {
      int kk = e % 8, mm = e / 8;
      int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < m && gk < k) ? load_op(A, lda, gm, gk, opA) : cplx<T>{0, 0};
      int nn = e % 64, kb = e / 64;
      int gn = n0 + nn, gk2 = k0 + kb;
      Bs[kb][nn] = (gn < n && gk2 < k) ? load_op(B, ldb, gk2, gn, opB) : cplx<T>{0, 0};
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      cplx<T> a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = cfma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
      if (gm < m && gn < n) {
        cplx<T>* c = C + (long long)gm * ldc + gn;
        cplx<T> v = cmul(alpha, acc[i][j]);
        if (beta.re != (T)0 || beta.im != (T)0) v = cfma(beta, *c, v);
        *c = v;
      }
    }
}

// ---------------------------------------------------------------------------------------------
// FP32 complex GEMM for op(A) = A, op(B) = B (row-major, batched): C = alpha A B + beta C.
// 80x80 tile (N = 400 = 5 tiles), 256 threads as 16 x 16, 5 x 5 outputs per thread (rows
// ty + 16 i, columns tx + 16 j), K chunk 16 double-buffered through registers. The A tile is
// stored K-major with a row pitch of 81 complex so that the 16 threads filling one A row write
// 16 distinct bank pairs.
// ---------------------------------------------------------------------------------------------
constexpr int CG_T = 80, CG_K = 16, CG_AP = 81;

__global__ void __launch_bounds__(256, 2) k_cgemm_nn(int m, int n, int k, c64 alpha, const c64* __restrict__ A,
                                                    long long lda, long long sA, const c64* __restrict__ B,
                                                    long long ldb, long long sB, c64 beta, c64* __restrict__ C,
                                                    long long ldc, long long sC) {
  __shared__ float2 As[2][CG_K][CG_AP];
  __shared__ float2 Bs[2][CG_K][CG_T];
  const int bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int m0 = blockIdx.y * CG_T, n0 = blockIdx.x * CG_T;
  const int t = threadIdx.x, tx = t % 16, ty = t / 16;
  // global -> register staging: 5 A elements (row e / 16, k e % 16) and 5 B elements
  // (k e / 80, column e % 80) for e = t + 256 c
  float2 ra[5], rb[5];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const int e = t + 256 * c;
      const int ar = m0 + e / CG_K, ak = k0 + e % CG_K;
      ra[c] = (ar < m && ak < k) ? *reinterpret_cast<const float2*>(A + (long long)ar * lda + ak) : make_float2(0.f, 0.f);
      const int bk = k0 + e / CG_T, bc = n0 + e % CG_T;
      rb[c] = (bk < k && bc < n) ? *reinterpret_cast<const float2*>(B + (long long)bk * ldb + bc) : make_float2(0.f, 0.f);
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const int e = t + 256 * c;
      As[buf][e % CG_K][e / CG_K] = ra[c];
      Bs[buf][e / CG_T][e % CG_T] = rb[c];
    }
  };
  float2 acc[5][5];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < 5; ++j) acc[i][j] = make_float2(0.f, 0.f);
  fetch(0);
  stash(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < k; k0 += CG_K) {
    const bool more = k0 + CG_K < k;
    if (more) fetch(k0 + CG_K);
#pragma unroll
    for (int kk = 0; kk < CG_K; ++kk) {
      float2 a[5], b[5];
#pragma unroll
      for (int i = 0; i < 5; ++i) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 5; ++j) b[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j < 5; ++j) {
          acc[i][j].x = fmaf(a[i].x, b[j].x, acc[i][j].x);
          acc[i][j].x = fmaf(-a[i].y, b[j].y, acc[i][j].x);
          acc[i][j].y = fmaf(a[i].x, b[j].y, acc[i][j].y);
          acc[i][j].y = fmaf(a[i].y, b[j].x, acc[i][j].y);
        }
    }
    if (more) {
      stash(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
  const bool use_beta = beta.re != 0.f || beta.im != 0.f;
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      const int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
      if (gm < m && gn < n) {
        c64* c = C + (long long)gm * ldc + gn;
        c64 v = cmul(alpha, c64{acc[i][j].x, acc[i][j].y});
        if (use_beta) v = cfma(beta, *c, v);
        *c = v;
      }
    }
}

template <typename T>
void launch_zgemm(int m, int n, int k, cplx<T> alpha, const cplx<T>* A, long long lda, long long sA, Op opA,
                  const cplx<T>* B, long long ldb, long long sB, Op opB, cplx<T> beta, cplx<T>* C, long long ldc,
                  long long sC, int batch, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (opA == OP_N && opB == OP_N) {
      dim3 grid((n + CG_T - 1) / CG_T, (m + CG_T - 1) / CG_T, batch);
      ++::gw::g_launch_count, k_cgemm_nn<<<grid, 256, 0, st>>>(m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC);
      return;
    }
  }
  dim3 grid((n + 63) / 64, (m + 63) / 64, batch);
  ++::gw::g_launch_count, k_zgemm<T><<<grid, 256, 0, st>>>(m, n, k, alpha, A, lda, sA, (int)opA, B, ldb, sB, (int)opB, beta, C, ldc, sC);
}
template void launch_zgemm<double>(int, int, int, c128, const c128*, long long, long long, Op, const c128*,
                                   long long, long long, Op, c128, c128*, long long, long long, int, cudaStream_t);
template void launch_zgemm<float>(int, int, int, c64, const c64*, long long, long long, Op, const c64*, long long,
                                  long long, Op, c64, c64*, long long, long long, int, cudaStream_t);

// ---------------------------------------------------------------------------------------------
// chi0 on CUDA cores (the FP64 method): Hermitian weighted rank-K update, lower tiles only,
// one block per (lower 32x32 tile, frequency).
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_chi0_simt(int N, int K, const cplx<T>* __restrict__ Mt, long long ldm,
                                                   const float* __restrict__ delta_f,
                                                   const double* __restrict__ delta_d,
                                                   const double* __restrict__ freq, double scale,
                                                   c128* __restrict__ chi0) {
  __shared__ cplx<T> As[16][33];
  __shared__ cplx<T> Bs[16][33];
  // lower-tile index -> (ti, tj), ti >= tj
  int t = blockIdx.x;
  int ti = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
  while (ti * (ti + 1) / 2 > t) --ti;
  int tj = t - ti * (ti + 1) / 2;
  const int w_i = blockIdx.y;
  const T om = (T)freq[w_i];
  const int mu0 = ti * 32, nu0 = tj * 32;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  cplx<T> acc[2][2] = {{{0, 0}, {0, 0}}, {{0, 0}, {0, 0}}};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * 32; e += 256) {
      int kk = e % 16, mm = e / 16;
      int gk = k0 + kk;
      cplx<T> a = {0, 0}, b = {0, 0};
      if (gk < K) {
        T d = delta_d ? (T)delta_d[gk] : (T)delta_f[gk];
        T w = (T)2 * d / (om * om + d * d);
        if (mu0 + mm < N) {
          a = Mt[(long long)(mu0 + mm) * ldm + gk];
          a.re *= w;
          a.im *= w;
        }
        if (nu0 + mm < N) b = Mt[(long long)(nu0 + mm) * ldm + gk];
      }
      As[kk][mm] = a;
      Bs[kk][mm] = b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      cplx<T> a0 = As[kk][ty], a1 = As[kk][ty + 16];
      cplx<T> b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
      // a * conj(b)
      acc[0][0] = cadd(acc[0][0], cmulc(a0, b0));
      acc[0][1] = cadd(acc[0][1], cmulc(a0, b1));
      acc[1][0] = cadd(acc[1][0], cmulc(a1, b0));
      acc[1][1] = cadd(acc[1][1], cmulc(a1, b1));
    }
    __syncthreads();
  }
  c128* out = chi0 + (long long)w_i * N * N;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      int mu = mu0 + ty + 16 * i, nu = nu0 + tx + 16 * j;
      if (mu < N && nu < N && (ti != tj || mu >= nu)) {
        double re = scale * (double)acc[i][j].re, im = scale * (double)acc[i][j].im;
        c128* p = out + (long long)mu * N + nu;
        p->re += re;
        p->im += im;
        if (mu != nu) {
          c128* q = out + (long long)nu * N + mu;
          q->re += re;
          q->im -= im;
        }
      }
    }
}

template <typename T>
void launch_chi0_simt(int N, int K, const cplx<T>* Mt, long long ldm, const float* delta_f, const double* delta_d,
                      const double* freq, int nw, double scale, c128* chi0, cudaStream_t st) {
  int nt = (N + 31) / 32;
  dim3 grid(nt * (nt + 1) / 2, nw);
  ++::gw::g_launch_count, k_chi0_simt<T><<<grid, 256, 0, st>>>(N, K, Mt, ldm, delta_f, delta_d, freq, scale, chi0);
}
template void launch_chi0_simt<double>(int, int, const c128*, long long, const float*, const double*, const double*,
                                       int, double, c128*, cudaStream_t);
template void launch_chi0_simt<float>(int, int, const c64*, long long, const float*, const double*, const double*,
                                      int, double, c128*, cudaStream_t);

// ---------------------------------------------------------------------------------------------
// FP64 Cholesky factorisation and inversion of eps~ (Hermitian positive definite), one block
// per matrix:
//   1) eps~ = U^H U, up-looking, U in place in the upper triangle;
//   2) W = U^{-1} (upper) by backward substitution into the work buffer;
//   3) A := W W^H - I (= eps~^{-1} - I), lower 32 x 32 tiles from shared-memory K chunks, mirrored.
// The dot products of one step of 1) and 2) have lengths up to N while only N - j of them exist,
// so each is split over P threads (k strided, P = threads / dots, at least 16 terms per part) and
// the parts are combined in shared memory: the late steps, few long dots, run in parallel.
// ---------------------------------------------------------------------------------------------
constexpr int CHOL_THREADS = 512;
constexpr int CHOL_T = 32, CHOL_TP = CHOL_T + 1;   // phase-3 tile and its row pitch (complex)

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0;
  if (threadIdx.x < 32) {
    s = (threadIdx.x < blockDim.x / 32) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) red[0] = s;
  }
  __syncthreads();
  s = red[0];
  __syncthreads();
  return s;
}

// s += conj(c) u and s += u w as explicit fused multiply-adds (4 DFMA per complex product; the
// unfused a*b + c*d form costs a multiply, a fused multiply-add and an add per pair)
__device__ __forceinline__ void chol_cmac_conj(c128 c, c128 u, double& sr, double& si) {
  sr = fma(c.im, u.im, fma(c.re, u.re, sr));
  si = fma(-c.im, u.re, fma(c.re, u.im, si));
}
__device__ __forceinline__ void chol_cmac(c128 u, c128 w, double& sr, double& si) {
  sr = fma(-u.im, w.im, fma(u.re, w.re, sr));
  si = fma(u.im, w.re, fma(u.re, w.im, si));
}

// parts per dot: n dots of length up to len over `threads` threads
__device__ __forceinline__ int chol_parts(int n, int len, int threads) {
  if (n <= 0) return 1;
  return max(1, min(threads / n, len / 16));
}

size_t chol_smem_bytes(int N) {
  return sizeof(c128) * std::max<size_t>((size_t)N + CHOL_THREADS, (size_t)2 * CHOL_T * CHOL_TP);
}

__global__ void __launch_bounds__(CHOL_THREADS) k_chol_inv(int N, c128* __restrict__ Aall, long long stride,
                                                           c128* __restrict__ Wall, int* __restrict__ status) {
  extern __shared__ c128 dyn[];
  c128* col = dyn;                   // [N]: the current column (1) or row (2) of U
  c128* part = dyn + N;              // [CHOL_THREADS]: partial dot products
  __shared__ double red[32];
  __shared__ double s_piv;
  const int t = threadIdx.x, bd = blockDim.x;
  c128* A = Aall + blockIdx.x * stride;
  c128* W = Wall + blockIdx.x * stride;
  // 1) eps~ = U^H U: U[j][i] = (A[j][i] - sum_{k<j} conj(U[k][j]) U[k][i]) / U[j][j]
  for (int j = 0; j < N; ++j) {
    for (int k = t; k < j; k += bd) col[k] = A[(long long)k * N + j];
    __syncthreads();
    double pp = 0;
    for (int k = t; k < j; k += bd) pp = fma(col[k].im, col[k].im, fma(col[k].re, col[k].re, pp));
    const double s = block_sum(pp, red);
    if (t == 0) {
      double piv = A[(long long)j * N + j].re - s;
      if (!(piv > 0.0)) {
        atomicOr(status, ST_NOT_PD);
        piv = 1.0;
      }
      s_piv = sqrt(piv);
      A[(long long)j * N + j] = c128{s_piv, 0.0};
    }
    __syncthreads();
    const double inv = 1.0 / s_piv;
    const int R = N - j - 1;                    // rows i = j + 1 .. N - 1
    const int P = chol_parts(R, j, bd);
    if (P == 1) {
      for (int i = j + 1 + t; i < N; i += bd) {
        double sr = 0, si = 0;
        for (int k = 0; k < j; ++k) {
          const c128 u = A[(long long)k * N + i], c = col[k];
          chol_cmac_conj(c, u, sr, si);
        }
        const c128 a = A[(long long)j * N + i];
        A[(long long)j * N + i] = c128{(a.re - sr) * inv, (a.im - si) * inv};
      }
    } else {
      double sr = 0, si = 0;
      if (t < R * P) {
        const int i = j + 1 + t % R;
        for (int k = t / R; k < j; k += P) {
          const c128 u = A[(long long)k * N + i], c = col[k];
          chol_cmac_conj(c, u, sr, si);
        }
        part[t] = c128{sr, si};
      }
      __syncthreads();
      if (t < R) {
        for (int p = 1; p < P; ++p) {
          sr += part[p * R + t].re;
          si += part[p * R + t].im;
        }
        const int i = j + 1 + t;
        const c128 a = A[(long long)j * N + i];
        A[(long long)j * N + i] = c128{(a.re - sr) * inv, (a.im - si) * inv};
      }
    }
    __syncthreads();
  }
  // 2) W = U^{-1} (upper), rows from the bottom:
  //    W[i][i] = 1/U[i][i];  W[i][l] = -(1/U[i][i]) sum_{k=i+1}^{l} U[i][k] W[k][l]
  for (long long e = t; e < (long long)N * N; e += bd) W[e] = c128{0.0, 0.0};
  __syncthreads();
  for (int i = N - 1; i >= 0; --i) {
    for (int k = i + t; k < N; k += bd) col[k] = A[(long long)i * N + k];
    __syncthreads();
    const double dinv = 1.0 / col[i].re;
    const int R = N - i;                        // columns l = i .. N - 1
    const int P = chol_parts(R, R - 1, bd);
    if (P == 1) {
      for (int l = i + t; l < N; l += bd) {
        double sr = 0, si = 0;
        for (int k = i + 1; k <= l; ++k) {
          const c128 u = col[k], w = W[(long long)k * N + l];
          chol_cmac(u, w, sr, si);
        }
        W[(long long)i * N + l] = (l == i) ? c128{dinv, 0.0} : c128{-sr * dinv, -si * dinv};
      }
    } else {
      double sr = 0, si = 0;
      if (t < R * P) {
        const int l = i + t % R;
        for (int k = i + 1 + t / R; k <= l; k += P) {
          const c128 u = col[k], w = W[(long long)k * N + l];
          chol_cmac(u, w, sr, si);
        }
        part[t] = c128{sr, si};
      }
      __syncthreads();
      if (t < R) {
        for (int p = 1; p < P; ++p) {
          sr += part[p * R + t].re;
          si += part[p * R + t].im;
        }
        const int l = i + t;
        W[(long long)i * N + l] = (l == i) ? c128{dinv, 0.0} : c128{-sr * dinv, -si * dinv};
      }
    }
    __syncthreads();
  }
  // 3) A = W W^H - I: A[i][l] = sum_{k >= max(i,l)} W[i][k] conj(W[l][k]) over lower tiles (ti >= tl);
  //    W[i][k] = 0 for k < i, so K starts at the tile row ti. Each thread owns the outputs
  //    (orow, oc) and (orow + 16, oc) of the tile.
  c128(*Ti)[CHOL_TP] = reinterpret_cast<c128(*)[CHOL_TP]>(dyn);
  c128(*Tl)[CHOL_TP] = reinterpret_cast<c128(*)[CHOL_TP]>(dyn + CHOL_T * CHOL_TP);
  const int nt = (N + CHOL_T - 1) / CHOL_T;
  const int oc = t % CHOL_T, orow = t / CHOL_T;   // orow < 16 with 512 threads
  for (int ti = 0; ti < nt; ++ti) {
    for (int tl = 0; tl <= ti; ++tl) {
      double s0r = 0, s0i = 0, s1r = 0, s1i = 0;
      for (int k0 = ti * CHOL_T; k0 < N; k0 += CHOL_T) {
        for (int e = t; e < 2 * CHOL_T * CHOL_T; e += bd) {
          const int which = e / (CHOL_T * CHOL_T), r = (e % (CHOL_T * CHOL_T)) / CHOL_T, c = e % CHOL_T;
          const int row = (which == 0 ? ti : tl) * CHOL_T + r, kk = k0 + c;
          const c128 v = (row < N && kk < N) ? W[(long long)row * N + kk] : c128{0.0, 0.0};
          if (which == 0) Ti[r][c] = v; else Tl[r][c] = v;
        }
        __syncthreads();
        if (orow < CHOL_T / 2) {
#pragma unroll 8
          for (int c = 0; c < CHOL_T; ++c) {
            const c128 b = Tl[oc][c], a0 = Ti[orow][c], a1 = Ti[orow + CHOL_T / 2][c];
            chol_cmac_conj(b, a0, s0r, s0i);      // a0 conj(b)
            chol_cmac_conj(b, a1, s1r, s1i);
          }
        }
        __syncthreads();
      }
      if (orow < CHOL_T / 2) {
        const int ll = tl * CHOL_T + oc;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int ii = ti * CHOL_T + orow + h * (CHOL_T / 2);
          double sr = h ? s1r : s0r, si = h ? s1i : s0i;
          if (ii < N && ll < N && ii >= ll) {
            if (ii == ll) {
              sr -= 1.0;
              si = 0.0;
            }
            A[(long long)ii * N + ll] = c128{sr, si};
            if (ii != ll) A[(long long)ll * N + ii] = c128{sr, -si};
          }
        }
      }
    }
  }
}

void launch_chol_inv_minus_I(int N, c128* A, int batch, long long stride, c128* work, int* status, cudaStream_t st) {
  const size_t smem = chol_smem_bytes(N);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_chol_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  ++::gw::g_launch_count, k_chol_inv<<<batch, CHOL_THREADS, smem, st>>>(N, A, stride, work, status);
}

// ---------------------------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_axpby_identity(int N, cplx<T>* A, long long s, T diag) {
  cplx<T>* a = A + blockIdx.y * s;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
    a[(long long)i * N + i].re += diag;
}
template <typename T> void launch_axpby_identity(int N, cplx<T>* A, long long s, int batch, T diag, cudaStream_t st) {
  dim3 grid((N + 255) / 256, batch);
  ++::gw::g_launch_count, k_axpby_identity<T><<<grid, 256, 0, st>>>(N, A, s, diag);
}
template void launch_axpby_identity<double>(int, c128*, long long, int, double, cudaStream_t);
template void launch_axpby_identity<float>(int, c64*, long long, int, float, cudaStream_t);

// X[b] = C[b] + d I and XH[b] = X[b]^H, rounded to FP32 (a product and its conjugate transpose,
// the latter the right operand of a later product on the tensor-core kernel, which multiplies by
// the conjugate transpose of the rows it is given); 32 x 32 tiles, the transposed tile through
// shared memory
__global__ void k_take_both(int N, const c128* __restrict__ C, long long s, float d, c64* __restrict__ X,
                            c64* __restrict__ XH) {
  __shared__ c128 tt[32][33];
  const c128* Cb = C + blockIdx.z * s;
  c64* xb = X + blockIdx.z * s;
  c64* hb = XH + blockIdx.z * s;
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int row = j0 + r, col = i0 + threadIdx.x;
    if (row < N && col < N) tt[r][threadIdx.x] = Cb[(long long)row * N + col];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + r, j = j0 + threadIdx.x;
    if (i < N && j < N) {
      const float dd = (i == j) ? d : 0.0f;
      const c128 a = Cb[(long long)i * N + j];
      const c128 t = tt[threadIdx.x][r];   // C[j][i]
      xb[(long long)i * N + j] = c64{(float)a.re + dd, (float)a.im};
      hb[(long long)i * N + j] = c64{(float)t.re + dd, -(float)t.im};
    }
  }
}
// dev = max over the batch of max(|Re T_ij - delta_ij|, |Im T_ij|) (as the bits of a non-negative
// float; *dev must hold 0 on entry)
__global__ void k_dev_identity(int N, const c64* __restrict__ T, long long total, unsigned* __restrict__ dev) {
  float m = 0.f;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long r = e % ((long long)N * N);
    const int i = (int)(r / N), j = (int)(r % N);
    const c64 v = T[e];
    m = fmaxf(m, fmaxf(fabsf(v.re - (i == j ? 1.0f : 0.0f)), fabsf(v.im)));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(dev, __float_as_uint(m));
}
void launch_dev_identity(int N, const c64* T, long long total, unsigned* dev, cudaStream_t st) {
  ++::gw::g_launch_count, k_dev_identity<<<(int)std::min<long long>((total + 255) / 256, 152LL * 8), 256, 0, st>>>(
      N, T, total, dev);
}

void launch_take_both(int N, const c128* C, long long s, int batch, float d, c64* X, c64* XH, cudaStream_t st) {
  dim3 grid((N + 31) / 32, (N + 31) / 32, batch);
  ++::gw::g_launch_count, k_take_both<<<grid, dim3(32, 8), 0, st>>>(N, C, s, d, X, XH);
}

__global__ void k_convert(int n, const c128* in, c64* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = c64{(float)in[i].re, (float)in[i].im};
}
void launch_convert(int n, const c128* in, c64* out, cudaStream_t st) {
  ++::gw::g_launch_count, k_convert<<<std::min((n + 255) / 256, 152 * 32), 256, 0, st>>>(n, in, out);
}

// Dominant eigenpair by power iteration with a Rayleigh quotient (one block, FP64). Each warp
// takes whole rows of A (coalesced along the row), the iterate stays in shared memory.
__global__ void __launch_bounds__(1024) k_power_iter(int N, const c128* __restrict__ A, c128* __restrict__ x,
                                                     double* lam, int iters) {
  extern __shared__ c128 v[];   // [2N]
  __shared__ double red[32];
  c128* y = v + N;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  for (int i = threadIdx.x; i < N; i += blockDim.x) v[i] = c128{1.0 + 0.001 * (i % 7), 0.0};
  __syncthreads();
  double rq = 0;
  int extra = 10;
  for (int it = 0; it < iters; ++it) {
    for (int i = warp; i < N; i += nwarp) {
      const c128* a = A + (long long)i * N;
      double sr = 0, si = 0;
      for (int j = lane; j < N; j += 32) {
        const c128 aa = a[j], b = v[j];
        sr = fma(aa.re, b.re, fma(-aa.im, b.im, sr));
        si = fma(aa.re, b.im, fma(aa.im, b.re, si));
      }
      for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
      }
      if (lane == 0) y[i] = c128{sr, si};
    }
    __syncthreads();
    double p = 0, d = 0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      p += y[i].re * y[i].re + y[i].im * y[i].im;
      d += v[i].re * y[i].re + v[i].im * y[i].im;   // Re v^H y
    }
    double nrm2 = block_sum(p, red);
    rq = block_sum(d, red);
    double inv = 1.0 / sqrt(nrm2);
    double dv = 0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const c128 nv = c128{y[i].re * inv, y[i].im * inv};
      dv += (nv.re - v[i].re) * (nv.re - v[i].re) + (nv.im - v[i].im) * (nv.im - v[i].im);
      v[i] = nv;
    }
    // converged: the step has shrunk geometrically below 1e-12; ten more steps (the dominant
    // eigenvalue is positive, so the iterate does not flip) take it to the rounding level
    const double step = sqrt(block_sum(dv, red));
    if (step < 1e-12) {
      if (extra == 0) break;
      --extra;
    }
  }
  // fix the phase: largest-magnitude component real positive
  if (threadIdx.x == 0) {
    int imax = 0;
    double best = -1;
    for (int i = 0; i < N; ++i) {
      double m = v[i].re * v[i].re + v[i].im * v[i].im;
      if (m > best) { best = m; imax = i; }
    }
    double m = sqrt(best);
    red[0] = v[imax].re / m;
    red[1] = -v[imax].im / m;
    *lam = rq;
  }
  __syncthreads();
  c128 ph = c128{red[0], red[1]};
  for (int i = threadIdx.x; i < N; i += blockDim.x) x[i] = cmul(v[i], ph);
}
void launch_power_iter(int N, const c128* A, c128* x, double* lam, int iters, cudaStream_t st) {
  const int smem = 2 * N * (int)sizeof(c128);   // above 48 KB from N = 1536 on: opt in
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_power_iter, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  ++::gw::g_launch_count, k_power_iter<<<1, 1024, smem, st>>>(N, A, x, lam, iters);
}

__global__ void k_rank1(int N, c128* A, const c128* x, double alpha) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)N * N;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / N), j = (int)(e % N);
    c128 v = cmulc(x[i], x[j]);
    A[e].re += alpha * v.re;
    A[e].im += alpha * v.im;
  }
}
void launch_rank1(int N, c128* A, const c128* x, double alpha, cudaStream_t st) {
  ++::gw::g_launch_count, k_rank1<<<std::min((N * N + 255) / 256, 152 * 16), 256, 0, st>>>(N, A, x, alpha);
}

// head[w] += pref * sum_r |pq_r|^2 2 / (D (D^2 + w^2));  h[w][nu] += sum_r conj(pq_r) Mt[nu][r] 2/(w^2 + D^2)
template <typename T>
__global__ void k_head_wings(int N, int K, const cplx<T>* __restrict__ Mt, long long ldm,
                             const double* __restrict__ delta, const c128* __restrict__ pq,
                             const double* __restrict__ freq, double head_pref, double* head, c128* h) {
  __shared__ double red[32];
  const int nu = blockIdx.x, w_i = blockIdx.y;
  const double om = freq[w_i];
  if (nu == N) {  // one extra block row computes the head
    double part = 0;
    for (int r = threadIdx.x; r < K; r += blockDim.x) {
      double d = delta[r];
      c128 p = pq[r];
      part += (p.re * p.re + p.im * p.im) * 2.0 / (d * (d * d + om * om));
    }
    double s = block_sum(part, red);
    if (threadIdx.x == 0) head[w_i] += head_pref * s;
    return;
  }
  double sr = 0, si = 0;
  for (int r = threadIdx.x; r < K; r += blockDim.x) {
    double d = delta[r];
    double wt = 2.0 / (om * om + d * d);
    c128 p = pq[r];
    cplx<T> m = Mt[(long long)nu * ldm + r];
    // conj(p) * m
    sr += wt * (p.re * (double)m.re + p.im * (double)m.im);
    si += wt * (p.re * (double)m.im - p.im * (double)m.re);
  }
  double a = block_sum(sr, red);
  double b = block_sum(si, red);
  if (threadIdx.x == 0) {
    h[(long long)w_i * N + nu].re += a;
    h[(long long)w_i * N + nu].im += b;
  }
}
template <typename T>
void launch_head_wings(int N, int K, const cplx<T>* Mt, long long ldm, const double* delta, const c128* pq,
                       const double* freq, int nw, double head_pref, double* head, c128* h, cudaStream_t st) {
  dim3 grid(N + 1, nw);
  ++::gw::g_launch_count, k_head_wings<T><<<grid, 256, 0, st>>>(N, K, Mt, ldm, delta, pq, freq, head_pref, head, h);
}
template void launch_head_wings<double>(int, int, const c128*, long long, const double*, const c128*, const double*,
                                        int, double, double*, c128*, cudaStream_t);
template void launch_head_wings<float>(int, int, const c64*, long long, const double*, const c128*, const double*, int,
                                       double, double*, c128*, cudaStream_t);

// Pair tables for rows r = ((kk*na)+a)*nb+b (a at k+q, b at k, k = kk0+kk):
// delta[r] = eps_a(k+q) - eps_b(k); pq[r] = (p(k) . qhat)_{b a} (used at q = 0 only).
__global__ void k_pairs(int NBd, int n1, int n2, int n3, int q, int kk0, int nkk, int a0, int na, int b0, int nb,
                        const double* __restrict__ eps, const c128* __restrict__ pmom, double qx, double qy,
                        double qz, double* delta, float* delta_f, c128* pq) {
  const long long total = (long long)nkk * na * nb;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < total;
       r += (long long)gridDim.x * blockDim.x) {
    int b = (int)(r % nb), a = (int)((r / nb) % na), kk = (int)(r / ((long long)na * nb));
    int k = kk0 + kk;
    int k3 = k % n3, k2 = (k / n3) % n2, k1 = k / (n2 * n3);
    int q3 = q % n3, q2 = (q / n3) % n2, q1 = q / (n2 * n3);
    int kq = (((k1 + q1) % n1) * n2 + ((k2 + q2) % n2)) * n3 + ((k3 + q3) % n3);
    double d = eps[(long long)kq * NBd + a0 + a] - eps[(long long)k * NBd + b0 + b];
    if (delta) delta[r] = d;
    if (delta_f) delta_f[r] = (float)d;
    if (pq) {
      c128 s = {0, 0};
      const double qh[3] = {qx, qy, qz};
      for (int x = 0; x < 3; ++x) {
        c128 p = pmom[(((long long)k * 3 + x) * NBd + (b0 + b)) * NBd + (a0 + a)];
        s.re += qh[x] * p.re;
        s.im += qh[x] * p.im;
      }
      pq[r] = s;
    }
  }
}
void launch_pairs(int NK, int NBd, const int* nk, int q, int kk0, int nkk, int a0, int na, int b0, int nb,
                  const double* eps, const c128* pmom, const double* qhat, double* delta, float* delta_f, c128* pq,
                  cudaStream_t st) {
  long long total = (long long)nkk * na * nb;
  int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 32);
  ++::gw::g_launch_count, k_pairs<<<blocks, 256, 0, st>>>(NBd, nk[0], nk[1], nk[2], q, kk0, nkk, a0, na, b0, nb, eps, pmom,
                                  qhat ? qhat[0] : 0, qhat ? qhat[1] : 0, qhat ? qhat[2] : 0, delta, delta_f, pq);
}

// eps~(0)[w] += (head_w - 1) x1 x1^H + x1 r_w + r_w^H x1^H,  r_w[nu] = -c conj(Vbh[w][nu])
__global__ void k_q0_correction(int N, c128* eps_t, const c128* __restrict__ x1, const c128* __restrict__ Vbh,
                                const double* __restrict__ head, double c) {
  const int w_i = blockIdx.y;
  const double hm1 = head[w_i] - 1.0;
  c128* E = eps_t + (long long)w_i * N * N;
  const c128* v = Vbh + (long long)w_i * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)N * N;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / N), j = (int)(e % N);
    c128 xx = cmulc(x1[i], x1[j]);                  // x1_i conj(x1_j)
    c128 rj = c128{-c * v[j].re, c * v[j].im};      // r_j = -c conj(v_j)
    c128 ri = c128{-c * v[i].re, c * v[i].im};
    c128 t1 = cmul(x1[i], rj);                      // x1_i r_j
    c128 t2 = cmulc(cconj(ri), x1[j]);              // conj(r_i) conj(x1_j)
    E[e].re += hm1 * xx.re + t1.re + t2.re;
    E[e].im += hm1 * xx.im + t1.im + t2.im;
  }
}
void launch_q0_correction(int N, int nw, c128* eps_t, const c128* x1, const c128* Vbh, const double* head, double c,
                          cudaStream_t st) {
  dim3 grid(std::min((N * N + 255) / 256, 256), nw);
  ++::gw::g_launch_count, k_q0_correction<<<grid, 256, 0, st>>>(N, eps_t, x1, Vbh, head, c);
}

// Direction-averaged head and wings at q -> 0 (head_wings = 2).
// Cartesian pieces, accumulated over pair rows (all k): the head tensor
//   A6[w] = pref sum_r 2 Re(conj(p_a) p_b) / (D (D^2 + w^2)),  (a, b) = xx, yy, zz, xy, xz, yz,
// and the wing vectors h3[w][a][nu] = sum_r conj(p_a,r) M^nu_r 2 / (w^2 + D^2), pq3[a][r] = p_a(k)_{ia}.
constexpr int HW3_NB = 8;   // wing rows nu per block: the weight and the p_a(r) loads serve all of them

// Grid (nw, ceil(N / HW3_NB) + 1): the frequency varies fastest, so the blocks that read the same
// rows of M run together and share them in L2; the last row of blocks computes A6.
template <typename T>
__global__ void __launch_bounds__(256) k_head_wings3(int N, int K, const cplx<T>* __restrict__ Mt, long long ldm,
                                                     const double* __restrict__ delta, const c128* __restrict__ pq3,
                                                     long long ldp, const double* __restrict__ freq, double pref,
                                                     double* A6, c128* h3) {
  __shared__ double red[32];
  const int w_i = blockIdx.x;
  const double om = freq[w_i];
  if ((int)blockIdx.y * HW3_NB >= N) {
    double part[6] = {0, 0, 0, 0, 0, 0};
    for (int r = threadIdx.x; r < K; r += blockDim.x) {
      const double d = delta[r];
      const double f = 2.0 / (d * (d * d + om * om));
      const c128 px = pq3[r], py = pq3[ldp + r], pz = pq3[2 * ldp + r];
      part[0] += f * (px.re * px.re + px.im * px.im);
      part[1] += f * (py.re * py.re + py.im * py.im);
      part[2] += f * (pz.re * pz.re + pz.im * pz.im);
      part[3] += f * (px.re * py.re + px.im * py.im);
      part[4] += f * (px.re * pz.re + px.im * pz.im);
      part[5] += f * (py.re * pz.re + py.im * pz.im);
    }
    for (int c = 0; c < 6; ++c) {
      const double sc = block_sum(part[c], red);
      if (threadIdx.x == 0) A6[w_i * 6 + c] += pref * sc;
    }
    return;
  }
  const int nu0 = blockIdx.y * HW3_NB;
  const int nv = min(HW3_NB, N - nu0);
  double sr[HW3_NB][3], si[HW3_NB][3];
#pragma unroll
  for (int u = 0; u < HW3_NB; ++u)
#pragma unroll
    for (int a = 0; a < 3; ++a) sr[u][a] = si[u][a] = 0.0;
  for (int r = threadIdx.x; r < K; r += blockDim.x) {
    const double d = delta[r];
    const double wt = 2.0 / (om * om + d * d);
    c128 pw[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const c128 pp = pq3[a * ldp + r];
      pw[a] = c128{wt * pp.re, wt * pp.im};
    }
#pragma unroll
    for (int u = 0; u < HW3_NB; ++u) {
      if (u < nv) {
        const cplx<T> m = Mt[(long long)(nu0 + u) * ldm + r];
        const double mr = (double)m.re, mi = (double)m.im;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          sr[u][a] += pw[a].re * mr + pw[a].im * mi;
          si[u][a] += pw[a].re * mi - pw[a].im * mr;
        }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < HW3_NB; ++u) {
    if (u < nv) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double x = block_sum(sr[u][a], red);
        const double y = block_sum(si[u][a], red);
        if (threadIdx.x == 0) {
          c128& o = h3[((long long)w_i * 3 + a) * N + nu0 + u];
          o.re += x;
          o.im += y;
        }
      }
    }
  }
}
template <typename T>
void launch_head_wings3(int N, int K, const cplx<T>* Mt, long long ldm, const double* delta, const c128* pq3,
                        long long ldp, const double* freq, int nw, double pref, double* A6, c128* h3,
                        cudaStream_t st) {
  dim3 grid(nw, (N + HW3_NB - 1) / HW3_NB + 1);
  ++::gw::g_launch_count, k_head_wings3<T><<<grid, 256, 0, st>>>(N, K, Mt, ldm, delta, pq3, ldp, freq, pref, A6, h3);
}
template void launch_head_wings3<double>(int, int, const c128*, long long, const double*, const c128*, long long,
                                         const double*, int, double, double*, c128*, cudaStream_t);
template void launch_head_wings3<float>(int, int, const c64*, long long, const double*, const c128*, long long,
                                        const double*, int, double, double*, c128*, cudaStream_t);

// Per frequency w (one block): with y_a = Y[w][a][:] and g_b = y_b + Xb[w] y_b (G[w][nu][b] holds
// Xb y_b on entry), Gamma_ab = y_a^H g_b; the quadratic form of the Schur complement
//   s(q^) = 1 + q^T (A - Re Gamma) q,
// averaged over the direction rule (dirs [nd][4]: x, y, z, weight):
//   m[w] = { <1/s>, <q_a/s> (3), <q_a q_b/s> (xx, yy, zz, xy, xz, yz) }.
// G is completed to g in place. A non-positive s sets ST_NOT_PD.
__global__ void k_q0avg_moments(int N, const c128* __restrict__ Y, c128* G, const double* __restrict__ A6,
                                const double* __restrict__ dirs, int nd, double* m, int* status) {
  __shared__ double red[32];
  __shared__ double L[6];
  const int w_i = blockIdx.x;
  const c128* y = Y + (long long)w_i * 3 * N;
  c128* g = G + (long long)w_i * 3 * N;
  double gam[6] = {0, 0, 0, 0, 0, 0};
  const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
  for (int nu = threadIdx.x; nu < N; nu += blockDim.x) {
    c128 gv[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const c128 yb = y[b * N + nu];
      gv[b] = c128{g[nu * 3 + b].re + yb.re, g[nu * 3 + b].im + yb.im};
      g[nu * 3 + b] = gv[b];
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const c128 ya = y[ia[c] * N + nu];
      gam[c] += ya.re * gv[ib[c]].re + ya.im * gv[ib[c]].im;   // Re conj(y_a) g_b
    }
  }
  for (int c = 0; c < 6; ++c) {
    const double v = block_sum(gam[c], red);
    if (threadIdx.x == 0) L[c] = A6[w_i * 6 + c] - v;
  }
  __syncthreads();
  double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int d = threadIdx.x; d < nd; d += blockDim.x) {
    const double x = dirs[4 * d], yv = dirs[4 * d + 1], z = dirs[4 * d + 2], wt = dirs[4 * d + 3];
    const double sq = 1.0 + L[0] * x * x + L[1] * yv * yv + L[2] * z * z +
                      2.0 * (L[3] * x * yv + L[4] * x * z + L[5] * yv * z);
    if (!(sq > 0.0)) atomicOr(status, ST_NOT_PD);
    const double f = wt / sq;
    acc[0] += f;
    acc[1] += f * x;
    acc[2] += f * yv;
    acc[3] += f * z;
    acc[4] += f * x * x;
    acc[5] += f * yv * yv;
    acc[6] += f * z * z;
    acc[7] += f * x * yv;
    acc[8] += f * x * z;
    acc[9] += f * yv * z;
  }
  for (int c = 0; c < 10; ++c) {
    const double v = block_sum(acc[c], red);
    if (threadIdx.x == 0) m[w_i * 10 + c] = v;
  }
}
void launch_q0avg_moments(int N, int nw, const c128* Y, c128* G, const double* A6, const double* dirs, int nd,
                          double* m, int* status, cudaStream_t st) {
  ++::gw::g_launch_count, k_q0avg_moments<<<nw, 256, 0, st>>>(N, Y, G, A6, dirs, nd, m, status);
}

// X[w] += (m0 - 1) x1 x1^H - sum_a m1_a (x1 g_a^H + g_a x1^H) + sum_ab m2_ab g_a g_b^H
// (the direction average of eps~^-1 - 1 from the inverse of the body, Schur-complement form)
__global__ void k_q0avg_update(int N, int nw, c128* X, long long sX, const c128* __restrict__ x1,
                               const c128* __restrict__ G, const double* __restrict__ m) {
  const int w_i = blockIdx.y;
  const double* mm = m + w_i * 10;
  const double m2[3][3] = {{mm[4], mm[7], mm[8]}, {mm[7], mm[5], mm[9]}, {mm[8], mm[9], mm[6]}};
  const c128* g = G + (long long)w_i * 3 * N;
  c128* Xw = X + (long long)w_i * sX;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)N * N;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / N), j = (int)(e % N);
    const c128 xi = x1[i], xj = x1[j];
    c128 v = cmulc(xi, xj);
    v.re *= mm[0] - 1.0;
    v.im *= mm[0] - 1.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const c128 t = cadd(cmulc(xi, g[j * 3 + a]), cmulc(g[i * 3 + a], xj));
      v.re -= mm[1 + a] * t.re;
      v.im -= mm[1 + a] * t.im;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const c128 u = cmulc(g[i * 3 + a], g[j * 3 + b]);
        v.re += m2[a][b] * u.re;
        v.im += m2[a][b] * u.im;
      }
    }
    Xw[e].re += v.re;
    Xw[e].im += v.im;
  }
}
void launch_q0avg_update(int N, int nw, c128* X, long long sX, const c128* x1, const c128* G, const double* m,
                         cudaStream_t st) {
  dim3 grid(std::min((N * N + 255) / 256, 256), nw);
  ++::gw::g_launch_count, k_q0avg_update<<<grid, 256, 0, st>>>(N, nw, X, sX, x1, G, m);
}

__global__ void k_midgap(int NK, int NBd, int nocc, const double* eps, double* mu) {
  __shared__ double hmax[256], lmin[256];
  double h = -1e300, l = 1e300;
  for (int k = threadIdx.x; k < NK; k += blockDim.x) {
    h = fmax(h, eps[(long long)k * NBd + nocc - 1]);
    l = fmin(l, eps[(long long)k * NBd + nocc]);
  }
  hmax[threadIdx.x] = h;
  lmin[threadIdx.x] = l;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      hmax[threadIdx.x] = fmax(hmax[threadIdx.x], hmax[threadIdx.x + s]);
      lmin[threadIdx.x] = fmin(lmin[threadIdx.x], lmin[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *mu = 0.5 * (hmax[0] + lmin[0]);
}
void launch_midgap(int NK, int NBd, int nocc, const double* eps, double* mu, cudaStream_t st) {
  ++::gw::g_launch_count, k_midgap<<<1, 256, 0, st>>>(NK, NBd, nocc, eps, mu);
}

}  // namespace gw
