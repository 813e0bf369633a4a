// Frequency compression of the chi0 contraction (split-precision path).
//
// chi0(w_j) = scale * sum_r W_jr m_r m_r^H with W_jr = 2 D_r / (w_j^2 + D_r^2) (Eq. chi0_matrix,
// Hermitised). The weight matrix W [nw][K] has a small numerical rank in j. With the row norms
// n_j, the Gram matrix of the normalised rows G^_jj' = (W W^T)_jj' / (n_j n_j') = U^ L U^T (FP64),
// the expansion E_jt = n_j U^_jt and the projection P_jt = U^_jt / n_j:
//   W_j ~ sum_{t<T} E_jt v_t,  v_t = sum_j P_jt W_j,
//   chi0(w_j) = sum_{t<T} E_jt C_t,  C_t = scale * sum_r v_tr m_r m_r^H.
// T is the smallest count whose per-frequency residual |W_j - sum_{t<T} E_jt v_t| / n_j, computed
// directly in FP64 over all pair rows, is within the tolerance for every j. So the tensor-core
// contraction runs over T weight rows instead of nw frequencies; the C_t are accumulated in FP64
// like chi0, and the expansion back to the frequencies is FP64.
#include "gw_internal.h"

#include <algorithm>

namespace gw {

namespace {

// G[j][j'] += sum_r W_jr W_j'r over the rows r < K of this chunk (FP64; stored as complex with
// zero imaginary part for the Hermitian eigensolver)
__global__ void __launch_bounds__(256) k_wgram(int K, int nw, const double* __restrict__ delta,
                                               const double* __restrict__ freq, c128* __restrict__ G) {
  __shared__ double wt[64][65];  // [j][row in tile]
  const int np = nw * nw;
  double acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0.0;
  for (int r0 = blockIdx.x * 64; r0 < K; r0 += gridDim.x * 64) {
    for (int e = threadIdx.x; e < nw * 64; e += blockDim.x) {
      const int j = e / 64, rr = e % 64;
      const int r = r0 + rr;
      double v = 0.0;
      if (r < K) {
        const double d = delta[r], w = freq[j];
        v = 2.0 * d / (w * w + d * d);
      }
      wt[j][rr] = v;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int pidx = threadIdx.x + 256 * i;
      if (pidx < np) {
        const int j = pidx / nw, jj = pidx % nw;
        double s = 0.0;
        for (int rr = 0; rr < 64; ++rr) s += wt[j][rr] * wt[jj][rr];
        acc[i] += s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int pidx = threadIdx.x + 256 * i;
    if (pidx < np) atomicAdd(&G[pidx].re, acc[i]);
  }
}

// normalised Gram: G^_jj' = G_jj' / (n_j n_j'), n_j = sqrt(G_jj) (one block per problem)
__global__ void k_wnorm(int nw, c128* __restrict__ G, double* __restrict__ nrm) {
  G += (long long)blockIdx.x * nw * nw;
  nrm += (long long)blockIdx.x * nw;
  __shared__ double n[64];
  for (int j = threadIdx.x; j < nw; j += blockDim.x) n[j] = sqrt(fmax(G[j * nw + j].re, 1e-300));
  __syncthreads();
  for (int e = threadIdx.x; e < nw * nw; e += blockDim.x) G[e].re /= n[e / nw] * n[e % nw];
  for (int j = threadIdx.x; j < nw; j += blockDim.x) nrm[j] = n[j];
}

// E_jt = n_j U^_jt, P_jt = U^_jt / n_j   (one block per problem)
__global__ void k_wproj(int nw, const c128* __restrict__ Uh, const double* __restrict__ nrm, double* __restrict__ E,
                        double* __restrict__ Pm) {
  const long long o = (long long)blockIdx.x * nw * nw;
  for (int e = threadIdx.x; e < nw * nw; e += blockDim.x) {
    const double n = nrm[(long long)blockIdx.x * nw + e / nw];
    E[o + e] = n * Uh[o + e].re;
    Pm[o + e] = Uh[o + e].re / n;
  }
}

// err[j][T] += sum_r (W_jr - sum_{t<T} E_jt v_tr)^2 for T = 0 .. nw, v_t = sum_j P_jt W_j.
// Tiles of 64 pair rows: W and v of the tile in shared memory; thread (j, grp) keeps the running
// residual of frequency j over its rows of the tile and its squares for every T in registers.
__global__ void __launch_bounds__(256) k_wresid(int K, int nw, const double* __restrict__ delta,
                                                const double* __restrict__ freq, const double* __restrict__ E,
                                                const double* __restrict__ Pm, double* __restrict__ err) {
  __shared__ double ws[64][65];  // [row][j]
  __shared__ double vs[64][65];  // [row][t]
  // residual phase: thread (j, grp) takes frequency j and rows grp, grp + ng, ... of the chunk, so
  // that ng * nw <= 256 threads are busy for every nw (not 64 of each 64-thread quarter)
  const int ng = blockDim.x / nw;
  const int j = threadIdx.x % nw, grp = threadIdx.x / nw;
  double acc[65];
#pragma unroll
  for (int T = 0; T < 65; ++T) acc[T] = 0.0;
  for (int r0 = blockIdx.x * 64; r0 < K; r0 += gridDim.x * 64) {
    for (int e = threadIdx.x; e < 64 * nw; e += blockDim.x) {
      const int rr = e / nw, jj = e % nw, r = r0 + rr;
      double v = 0.0;
      if (r < K) {
        const double d = delta[r];
        v = 2.0 * d / (freq[jj] * freq[jj] + d * d);
      }
      ws[rr][jj] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * nw; e += blockDim.x) {
      const int rr = e / nw, t = e % nw;
      double sv = 0.0;
      for (int jj = 0; jj < nw; ++jj) sv += Pm[jj * nw + t] * ws[rr][jj];
      vs[rr][t] = sv;
    }
    __syncthreads();
    if (grp < ng) {
      for (int rr = grp; rr < 64; rr += ng) {
        double res = ws[rr][j];
#pragma unroll
        for (int T = 0; T < 65; ++T) {
          if (T <= nw) {
            acc[T] += res * res;
            if (T < nw) res -= E[j * nw + T] * vs[rr][T];
          }
        }
      }
    }
    __syncthreads();
  }
  // the groups' sums meet in shared memory (ws is free now), then one global add per (j, T)
  double* red = &ws[0][0];
  for (int e = threadIdx.x; e < nw * (nw + 1); e += blockDim.x) red[e] = 0.0;
  __syncthreads();
  if (grp < ng) {
#pragma unroll
    for (int T = 0; T < 65; ++T)
      if (T <= nw) atomicAdd(&red[j * (nw + 1) + T], acc[T]);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nw * (nw + 1); e += blockDim.x) atomicAdd(&err[e], red[e]);
}

// v[t][r] = sum_j P[j][t] W_jr (FP64 sum, fp32 out) for t < T, r < Kpad (0 beyond K)
__global__ void k_wtab_compressed(int K, int Kpad, int nw, int T, const double* __restrict__ delta,
                                  const double* __restrict__ freq, const double* __restrict__ Pm,
                                  float* __restrict__ wtab) {
  // one pair row per thread, 8 weight rows at a time: each Lorentzian weight is evaluated
  // ceil(T / 8) times instead of T times (the sum over j runs in the same order)
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < Kpad;
       r += (long long)gridDim.x * blockDim.x) {
    const double d = r < K ? delta[r] : 0.0;
    for (int t0 = 0; t0 < T; t0 += 8) {
      double s[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) s[u] = 0.0;
      if (r < K) {
        for (int j = 0; j < nw; ++j) {
          const double w = freq[j];
          const double wt = 2.0 * d / (w * w + d * d);
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (t0 + u < T) s[u] += Pm[j * nw + t0 + u] * wt;
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (t0 + u < T) wtab[(long long)(t0 + u) * Kpad + r] = (float)s[u];
    }
  }
}

// chi0[j][e] += sum_t E[j][t] C[t][e]  for every frequency j and element e < NN
// chi0[j] += sum_t E_jt C_t, 16 frequencies per pass (register accumulators; the C rows are
// re-read once per pass, from L2)
__global__ void k_expand(int nw, int T, long long NN, const double* __restrict__ E, const c128* __restrict__ C,
                         c128* __restrict__ chi0) {
  constexpr int JB = 16;
  __shared__ double u[64 * 64];
  for (int e = threadIdx.x; e < nw * T; e += blockDim.x) u[e] = E[(e / T) * nw + (e % T)];
  __syncthreads();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < NN; e += (long long)gridDim.x * blockDim.x) {
    for (int j0 = 0; j0 < nw; j0 += JB) {
      double re[JB], im[JB];
#pragma unroll
      for (int jj = 0; jj < JB; ++jj) re[jj] = im[jj] = 0.0;
      for (int t = 0; t < T; ++t) {
        const c128 c = C[(long long)t * NN + e];
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) {
          const double w = (j0 + jj < nw) ? u[(j0 + jj) * T + t] : 0.0;
          re[jj] = fma(w, c.re, re[jj]);
          im[jj] = fma(w, c.im, im[jj]);
        }
      }
#pragma unroll
      for (int jj = 0; jj < JB; ++jj) {
        if (j0 + jj < nw) {
          c128 o = chi0[(long long)(j0 + jj) * NN + e];
          o.re += re[jj];
          o.im += im[jj];
          chi0[(long long)(j0 + jj) * NN + e] = o;
        }
      }
    }
  }
}

}  // namespace

void launch_wgram(int K, int nw, const double* delta, const double* freq, c128* G, cudaStream_t st) {
  const int blocks = std::max(1, std::min((K + 63) / 64, 152 * 2));
  ++g_launch_count, k_wgram<<<blocks, 256, 0, st>>>(K, nw, delta, freq, G);
}

void launch_wnorm(int nw, int batch, c128* G, double* nrm, cudaStream_t st) {
  ++g_launch_count, k_wnorm<<<batch, 256, 0, st>>>(nw, G, nrm);
}

void launch_wproj(int nw, int batch, const c128* Uh, const double* nrm, double* E, double* Pm, cudaStream_t st) {
  ++g_launch_count, k_wproj<<<batch, 256, 0, st>>>(nw, Uh, nrm, E, Pm);
}

void launch_wresid(int K, int nw, const double* delta, const double* freq, const double* E, const double* Pm,
                   double* err, cudaStream_t st) {
  const int blocks = std::max(1, std::min((K + 63) / 64, 152 * 2));
  ++g_launch_count, k_wresid<<<blocks, 256, 0, st>>>(K, nw, delta, freq, E, Pm, err);
}

void launch_wtab_compressed(int K, int Kpad, int nw, int T, const double* delta, const double* freq, const double* Pm,
                            float* wtab, cudaStream_t st) {
  ++g_launch_count, k_wtab_compressed<<<(unsigned)std::min<long long>(((long long)Kpad + 255) / 256, 152 * 32), 256, 0, st>>>(
      K, Kpad, nw, T, delta, freq, Pm, wtab);
}

void launch_expand(int nw, int T, long long NN, const double* E, const c128* C, c128* chi0, cudaStream_t st) {
  ++g_launch_count, k_expand<<<(unsigned)std::min<long long>((NN + 255) / 256, 152 * 8), 256, 0, st>>>(nw, T, NN, E, C,
                                                                                                     chi0);
}

}  // namespace gw
