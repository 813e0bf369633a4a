// Ritz modes of eps~(w_ref) - 1 and the surrogate's frequency reconstruction (the paper has no
// counterpart). Small dense problems (block width nb <= 64) run in one thread block with the
// matrix in shared memory, in FP64:
//   k_small_chol_linv  G = L L^H (Cholesky) and L^-1, for Cholesky-QR of the iteration block
//   k_small_jacobi     Hermitian H = Z diag(theta) Z^H by cyclic Jacobi with parallel ordering
// and the reconstruction of S_nm on the fine frequencies (k_sur_assemble).
#include "gw_internal.h"

#include <algorithm>
#include <cmath>

namespace gw {

namespace {

__device__ __forceinline__ c128 cz(double r, double i) { return c128{r, i}; }
__device__ __forceinline__ c128 mulc(c128 a, c128 b) { return c128{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ c128 conjc(c128 a) { return c128{a.re, -a.im}; }
__device__ __forceinline__ c128 subc(c128 a, c128 b) { return c128{a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ c128 addc(c128 a, c128 b) { return c128{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ c128 scal(double s, c128 a) { return c128{s * a.re, s * a.im}; }

// G (Hermitian [nb][nb], lower part read) = L L^H; writes Linv = L^-1 (lower, zeros above).
// One block per problem of a batch (consecutive [nb][nb] matrices).
// A pivot that is not positive sets ST_NOT_PD and is replaced by a tiny positive value.
__global__ void __launch_bounds__(256) k_small_chol_linv(int nb, const c128* __restrict__ G, c128* __restrict__ Linv,
                                                         int* __restrict__ status) {
  extern __shared__ c128 L[];
  const int t = threadIdx.x;
  G += (long long)blockIdx.x * nb * nb;
  Linv += (long long)blockIdx.x * nb * nb;
  for (int e = t; e < nb * nb; e += blockDim.x) L[e] = G[e];
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (t == 0) {
      double d = L[j * nb + j].re;
      if (!(d > 0.0)) {
        atomicOr(status, ST_NOT_PD);
        d = 1e-300;
      }
      L[j * nb + j] = cz(sqrt(d), 0.0);
    }
    __syncthreads();
    const double inv = 1.0 / L[j * nb + j].re;
    for (int i = j + 1 + t; i < nb; i += blockDim.x) L[i * nb + j] = scal(inv, L[i * nb + j]);
    __syncthreads();
    const int m = nb - j - 1;
    for (int e = t; e < m * m; e += blockDim.x) {
      const int i = j + 1 + e / m, k = j + 1 + e % m;
      if (k <= i) L[i * nb + k] = subc(L[i * nb + k], mulc(L[i * nb + j], conjc(L[k * nb + j])));
    }
    __syncthreads();
  }
  // column j of L^-1 by forward substitution (one thread per column)
  for (int j = t; j < nb; j += blockDim.x) {
    for (int i = 0; i < j; ++i) Linv[i * nb + j] = cz(0, 0);
    c128 x[64];
    x[j] = cz(1.0 / L[j * nb + j].re, 0.0);
    Linv[j * nb + j] = x[j];
    for (int i = j + 1; i < nb; ++i) {
      c128 s = cz(0, 0);
      for (int k = j; k < i; ++k) s = addc(s, mulc(L[i * nb + k], x[k]));
      x[i] = scal(-1.0 / L[i * nb + i].re, s);
      Linv[i * nb + j] = x[i];
    }
  }
}

// Eigen-decomposition of the Hermitian H [nb][nb] (nb <= 64) by cyclic Jacobi, rounds of
// disjoint pairs (circle ordering). Rotation of pair (p, q), c = A_pq = |c| u:
//   tau = (A_qq - A_pp) / (2|c|), t = sign(tau) / (|tau| + sqrt(1 + tau^2)), cs = 1/sqrt(1+t^2), sn = t cs,
//   G = [[cs, sn], [-sn conj(u), cs conj(u)]]:  A <- G^H A G,  Z <- Z G.
// Output: theta [nb] descending, Z columns in the same order. One block per problem of a batch.
__global__ void __launch_bounds__(256) k_small_jacobi(int nb, const c128* __restrict__ H, double* __restrict__ theta,
                                                      c128* __restrict__ Zout, int max_sweeps) {
  extern __shared__ c128 sm[];
  c128* A = sm;
  c128* Z = sm + nb * nb;
  H += (long long)blockIdx.x * nb * nb;
  Zout += (long long)blockIdx.x * nb * nb;
  theta += (long long)blockIdx.x * nb;
  __shared__ int sp[32], sq[32];
  __shared__ double scs[32], ssn[32];
  __shared__ c128 su[32];
  __shared__ double red[256];
  __shared__ int done;
  __shared__ int order[64];
  const int t = threadIdx.x;
  const int np = nb + (nb & 1), npairs = np / 2;
  for (int e = t; e < nb * nb; e += blockDim.x) {
    A[e] = H[e];
    Z[e] = cz(e / nb == e % nb ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int r = 0; r < np - 1; ++r) {
      if (t < npairs) {
        const int a = (t == 0) ? 0 : 1 + (t - 1 + r) % (np - 1);
        const int k2 = np - 1 - t;
        const int b = 1 + (k2 - 1 + r) % (np - 1);
        int p = min(a, b), q = max(a, b);
        double cs = 1.0, sn = 0.0;
        c128 u = cz(1, 0);
        if (q < nb) {
          const c128 c = A[p * nb + q];
          const double rr = sqrt(c.re * c.re + c.im * c.im);
          const double scale = fabs(A[p * nb + p].re) + fabs(A[q * nb + q].re);
          if (rr > 1e-300 && rr > 1e-18 * scale) {
            u = cz(c.re / rr, c.im / rr);
            const double tau = (A[q * nb + q].re - A[p * nb + p].re) / (2.0 * rr);
            const double tt = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            cs = 1.0 / sqrt(1.0 + tt * tt);
            sn = tt * cs;
          } else {
            p = -1;
          }
        } else {
          p = -1;
        }
        sp[t] = p;
        sq[t] = q;
        scs[t] = cs;
        ssn[t] = sn;
        su[t] = u;
      }
      __syncthreads();
      for (int e = t; e < npairs * nb; e += blockDim.x) {  // rows p, q: A <- G^H A
        const int k = e / nb, j = e % nb, p = sp[k];
        if (p < 0) continue;
        const int q = sq[k];
        const double cs = scs[k], sn = ssn[k];
        const c128 u = su[k];
        const c128 ap = A[p * nb + j], aq = A[q * nb + j];
        const c128 uaq = mulc(u, aq);
        A[p * nb + j] = subc(scal(cs, ap), scal(sn, uaq));
        A[q * nb + j] = addc(scal(sn, ap), scal(cs, uaq));
      }
      __syncthreads();
      for (int e = t; e < npairs * nb; e += blockDim.x) {  // columns p, q: A <- A G, Z <- Z G
        const int k = e / nb, i = e % nb, p = sp[k];
        if (p < 0) continue;
        const int q = sq[k];
        const double cs = scs[k], sn = ssn[k];
        const c128 uc = conjc(su[k]);
        c128 ap = A[i * nb + p], aq = mulc(uc, A[i * nb + q]);
        A[i * nb + p] = subc(scal(cs, ap), scal(sn, aq));
        A[i * nb + q] = addc(scal(sn, ap), scal(cs, aq));
        ap = Z[i * nb + p];
        aq = mulc(uc, Z[i * nb + q]);
        Z[i * nb + p] = subc(scal(cs, ap), scal(sn, aq));
        Z[i * nb + q] = addc(scal(sn, ap), scal(cs, aq));
      }
      __syncthreads();
    }
    // convergence: off-diagonal Frobenius norm relative to the whole
    double off = 0.0, tot = 0.0;
    for (int e = t; e < nb * nb; e += blockDim.x) {
      const double m2 = A[e].re * A[e].re + A[e].im * A[e].im;
      tot += m2;
      if (e / nb != e % nb) off += m2;
    }
    red[t] = off;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
      if (t < h) red[t] += red[t + h];
      __syncthreads();
    }
    const double off_s = red[0];
    __syncthreads();
    red[t] = tot;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
      if (t < h) red[t] += red[t + h];
      __syncthreads();
    }
    if (t == 0) done = (off_s <= 1e-28 * red[0]);
    __syncthreads();
    if (done) break;
  }
  if (t == 0) {  // order by descending eigenvalue (selection)
    for (int i = 0; i < nb; ++i) order[i] = i;
    for (int i = 0; i < nb; ++i) {
      int best = i;
      for (int j = i + 1; j < nb; ++j)
        if (A[order[j] * nb + order[j]].re > A[order[best] * nb + order[best]].re) best = j;
      const int tmp = order[i];
      order[i] = order[best];
      order[best] = tmp;
    }
  }
  __syncthreads();
  for (int k = t; k < nb; k += blockDim.x) theta[k] = A[order[k] * nb + order[k]].re;
  for (int e = t; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, k = e % nb;
    Zout[e] = Z[i * nb + order[k]];
  }
}

// d[l * ldd + c] = Re sum_i conj(U[i][l]) T_c[i][l], T_c = X_c U  ([nc][N][k], stride sT)
__global__ void k_mode_diag(int N, int k, const c128* __restrict__ U, const c128* __restrict__ T, long long sT,
                            float* __restrict__ d, int ldd, int c0) {
  const int l = blockIdx.x, c = blockIdx.y;
  __shared__ double red[256];
  double acc = 0.0;
  const c128* Tc = T + c * sT;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const c128 u = U[(long long)i * k + l], x = Tc[(long long)i * k + l];
    acc += u.re * x.re + u.im * x.im;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) d[(long long)l * ldd + c0 + c] = (float)red[0];
}

// network inputs: sig_l = |d_l(w_ref)| (1 if 0), x_l = d_l / sig_l   (rows of [rows][nc])
__global__ void k_sur_inputs(int rows, int nc, const float* __restrict__ d, float* __restrict__ x,
                             float* __restrict__ sig) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= rows) return;
  float s = fabsf(d[(long long)l * nc]);
  if (!(s > 0.f)) s = 1.f;
  sig[l] = s;
  for (int c = 0; c < nc; ++c) x[(long long)l * nc + c] = d[(long long)l * nc + c] / s;
}

// training features from the mode diagonal on the full grid d [rows][nw]: sig_l = |d_l(w_j0)|
// (1 if 0), x [rows][nc] = d(coarse)/sig, y [rows][nf] = d(fine)/sig  (jmap as in k_sur_assemble)
__global__ void k_sur_features(int rows, int nw, int j0, const int* __restrict__ jmap, const float* __restrict__ d,
                               int nc, int nf, float* __restrict__ x, float* __restrict__ y) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= rows) return;
  float s = fabsf(d[(long long)l * nw + j0]);
  if (!(s > 0.f)) s = 1.f;
  for (int j = 0; j < nw; ++j) {
    const int c = jmap[j];
    const float v = d[(long long)l * nw + j] / s;
    if (c >= 0) {
      if (x) x[(long long)l * nc + c] = v;
    } else if (y) {
      y[(long long)l * nf + (-c - 1)] = v;
    }
  }
}

// frequency moments of X [nw][NN]: gram[a][b] += sum_e Re(conj(X[c_a][e]) X[j_b][e]) for the
// coarse a < nc and b < nc + nf (b < nc: coarse index, else fine); blocks split e
__global__ void __launch_bounds__(256) k_freq_moments(int nw, long long NN, const c128* __restrict__ X,
                                                      const int* __restrict__ cidx, const int* __restrict__ fidx,
                                                      int nc, int nf, long long per_block, double* __restrict__ gram) {
  __shared__ c128 xs[32][64];
  const long long e0 = blockIdx.x * per_block, e1 = min(NN, e0 + per_block);
  const int npair = nc * (nc + nf);
  double acc[4] = {0, 0, 0, 0};  // pairs tid, tid + 256, ... (npair <= 64 * 16 = 1024)
  for (long long eb = e0; eb < e1; eb += 32) {
    const int ne = (int)min((long long)32, e1 - eb);
    for (int t = threadIdx.x; t < 32 * nw; t += blockDim.x) {
      const int r = t / nw, j = t % nw;
      xs[r][j] = (r < ne) ? X[(long long)j * NN + eb + r] : c128{0, 0};
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int pidx = threadIdx.x + 256 * i;
      if (pidx >= npair) break;
      const int a = pidx / (nc + nf), b = pidx % (nc + nf);
      const int ja = cidx[a], jb = b < nc ? cidx[b] : fidx[b - nc];
      double sacc = 0.0;
      for (int r = 0; r < ne; ++r) sacc += xs[r][ja].re * xs[r][jb].re + xs[r][ja].im * xs[r][jb].im;
      acc[i] += sacc;
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int pidx = threadIdx.x + 256 * i;
    if (pidx < npair) atomicAdd(&gram[pidx], acc[i]);
  }
}

// coef[l][m] = sig_l * g[l][m]
__global__ void k_sur_coef(int rows, int nf, const float* __restrict__ sig, const float* __restrict__ g,
                           float* __restrict__ coef) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)rows * nf) return;
  coef[e] = sig[e / nf] * g[e];
}

// S_full[r][j] for every grid frequency j: the computed S at coarse j, else
//   sum_c L[m][c] S_c[r][c] + sum_l |P[r][l]|^2 coef[l][m]   (m = position of j among the fine)
// jmap[j] = c >= 0 for coarse, -(m + 1) for fine.
template <typename T>
__global__ void k_sur_assemble(int R, int nc, int nw, int k, const int* __restrict__ jmap, const T* __restrict__ Sc,
                               const cplx<T>* __restrict__ P, const float* __restrict__ coef, int nf,
                               const float* __restrict__ L, T* __restrict__ S) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)R * nw) return;
  const int r = (int)(e / nw), j = (int)(e % nw);
  const int c = jmap[j];
  if (c >= 0) {
    S[e] = Sc[(long long)r * nc + c];
    return;
  }
  const int m = -c - 1;
  T acc = 0;
  for (int i = 0; i < nc; ++i) acc += (T)L[(long long)m * nc + i] * Sc[(long long)r * nc + i];
  for (int l = 0; l < k; ++l) {
    const cplx<T> p = P[(long long)r * k + l];
    acc += (p.re * p.re + p.im * p.im) * (T)coef[(long long)l * nf + m];
  }
  S[e] = acc;
}

}  // namespace

void launch_small_chol_linv(int nb, int batch, const c128* G, c128* Linv, int* status, cudaStream_t st) {
  const size_t sm = (size_t)nb * nb * sizeof(c128);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_small_chol_linv, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 64 * (int)sizeof(c128));
    attr = true;
  }
  ++g_launch_count, k_small_chol_linv<<<batch, 256, sm, st>>>(nb, G, Linv, status);
}

void launch_small_jacobi(int nb, int batch, const c128* H, double* theta, c128* Z, cudaStream_t st) {
  const size_t sm = 2 * (size_t)nb * nb * sizeof(c128);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_small_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 64 * 64 * (int)sizeof(c128));
    attr = true;
  }
  ++g_launch_count, k_small_jacobi<<<batch, 256, sm, st>>>(nb, H, theta, Z, 40);
}

void launch_mode_diag(int N, int k, int nc, const c128* U, const c128* T, long long sT, float* d, int ldd, int c0,
                      cudaStream_t st) {
  ++g_launch_count, k_mode_diag<<<dim3(k, nc), 256, 0, st>>>(N, k, U, T, sT, d, ldd, c0);
}

void launch_sur_inputs(int rows, int nc, const float* d, float* x, float* sig, cudaStream_t st) {
  ++g_launch_count, k_sur_inputs<<<(rows + 127) / 128, 128, 0, st>>>(rows, nc, d, x, sig);
}

void launch_sur_features(int rows, int nw, int j0, const int* jmap, const float* d, int nc, int nf, float* x,
                         float* y, cudaStream_t st) {
  ++g_launch_count, k_sur_features<<<(rows + 127) / 128, 128, 0, st>>>(rows, nw, j0, jmap, d, nc, nf, x, y);
}

void launch_freq_moments(int nw, long long NN, const c128* X, const int* cidx, const int* fidx, int nc, int nf,
                         double* gram, cudaStream_t st) {
  const long long per_block = std::max(256LL, (NN + 151) / 152);
  const int blocks = (int)((NN + per_block - 1) / per_block);
  ++g_launch_count, k_freq_moments<<<blocks, 256, 0, st>>>(nw, NN, X, cidx, fidx, nc, nf, per_block, gram);
}

void launch_sur_coef(int rows, int nf, const float* sig, const float* g, float* coef, cudaStream_t st) {
  const long long n = (long long)rows * nf;
  ++g_launch_count, k_sur_coef<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(rows, nf, sig, g, coef);
}

template <typename T>
void launch_sur_assemble(int R, int nc, int nw, int k, const int* jmap, const T* Sc, const cplx<T>* P,
                         const float* coef, int nf, const float* L, T* S, cudaStream_t st) {
  const long long n = (long long)R * nw;
  ++g_launch_count, k_sur_assemble<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(R, nc, nw, k, jmap, Sc, P, coef,
                                                                                   nf, L, S);
}
template void launch_sur_assemble<float>(int, int, int, int, const int*, const float*, const c64*, const float*, int,
                                         const float*, float*, cudaStream_t);
template void launch_sur_assemble<double>(int, int, int, int, const int*, const double*, const c128*, const float*,
                                          int, const float*, double*, cudaStream_t);

}  // namespace gw
