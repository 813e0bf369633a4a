// Step (a): LRI triple coefficients -> band-pair coefficients M^mu_{ab}(k, q).
//
// Eq. (AO_triple_split2): C~^mu_{ij}(k+q,k) = C~^{mu(0)}_{j(0),i(-k-q)} + C~^{mu(0)}_{i(0),j(k)},
// with C~_{i(0),j(R)}^{mu(0)} nonzero only for mu on the atom of i, and the
// Fourier sums of Eqs. (expan_coeff_FT1/2). Inserting this into Eq. (AO_MO_transform)
// and contracting the NAO index that is not on mu's atom first gives the
// half-transformed coefficients (computed once per k at plan time)
//     T1^mu_{ib}(k) = sum_R e^{i k.R} sum_j C~^{mu(0)}_{i(0),j(R)} c_{jb}(k),   i on atom(mu)
// and, because the stored C~(R) are real (real NAOs and ABFs), the second
// sector's transform is conj(T1). Then per (k, q):
//     M^mu_{ab}(k,q) = sum_{j in A(mu)} c_{jb}(k) conj(T1^mu_{ja}(k+q))
//                    + sum_{i in A(mu)} conj(c_{ia}(k+q)) T1^mu_{ib}(k),
// which is Eq. (AO_MO_transform) exactly, with n_b(A) instead of N_b terms per sum.
#include "gw_internal.h"
#include <cuda_bf16.h>

namespace gw {

template <typename T>
__global__ void k_lri_halfT(const __grid_constant__ LriGeom g, const double* __restrict__ ctil,
                            const c128* __restrict__ evec, cplx<T>* __restrict__ T1, int A) {
  const int nb_A = g.atom_nb[A], nx_A = g.atom_nx[A];
  const long long total = (long long)g.NK * nx_A * nb_A * g.NBd;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    int b = (int)(idx % g.NBd);
    long long t = idx / g.NBd;
    int i = (int)(t % nb_A);
    t /= nb_A;
    int mu = (int)(t % nx_A);
    int k = (int)(t / nx_A);
    int k3 = k % g.nk[2], k2 = (k / g.nk[2]) % g.nk[1], k1 = k / (g.nk[1] * g.nk[2]);
    double acc_re = 0.0, acc_im = 0.0;
    const c128* ck = evec + (long long)k * g.NB * g.NBd;
    for (int r = 0; r < g.nR; ++r) {
      // phase e^{2 pi i k.R}, k = mesh point + offset in fractional coordinates
      double ph = 2.0 * (((double)k1 / g.nk[0] + g.koff[0]) * g.R[r][0] + ((double)k2 / g.nk[1] + g.koff[1]) * g.R[r][1] +
                         ((double)k3 / g.nk[2] + g.koff[2]) * g.R[r][2]);
      double s, c;
      sincospi(ph, &s, &c);
      const double* crow = ctil + g.ctil_off[A] + (((long long)r * nx_A + mu) * nb_A + i) * g.NB;
      double sr = 0.0, si = 0.0;
      for (int j = 0; j < g.NB; ++j) {
        c128 cj = ck[(long long)j * g.NBd + b];
        sr = fma(crow[j], cj.re, sr);
        si = fma(crow[j], cj.im, si);
      }
      acc_re += c * sr - s * si;
      acc_im += c * si + s * sr;
    }
    T1[g.t_off[A] + idx] = cplx<T>{(T)acc_re, (T)acc_im};
  }
}

template <typename T>
void launch_lri_halfT(const LriGeom& g, const double* ctil, const c128* evec, cplx<T>* T1, cplx<T>* /*T2*/,
                      cudaStream_t st) {
  for (int A = 0; A < g.n_atoms; ++A) {
    long long total = (long long)g.NK * g.atom_nx[A] * g.atom_nb[A] * g.NBd;
    int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 64);
    ++::gw::g_launch_count, k_lri_halfT<T><<<blocks, 256, 0, st>>>(g, ctil, evec, T1, A);
  }
}
template void launch_lri_halfT<double>(const LriGeom&, const double*, const c128*, c128*, c128*, cudaStream_t);

// fp32 (split-precision plans): the same sums as batched complex GEMMs, one per lattice vector R,
//   T1[k] (+)= C~(R) [(mu,i)][j] . (e^{2 pi i k.R} c(k)) [j][b],   batched over k,
// with C~(R) real (zero imaginary part) and the phase folded into a copy of c(k).
namespace {

__global__ void k_real_to_c64(long long n, const double* __restrict__ x, c64* __restrict__ y) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    y[e] = c64{(float)x[e], 0.f};
}

// cR[k][j][b] = e^{2 pi i k.R_r} c(k)[j][b] (phase in FP64)
__global__ void k_phase_evec(const __grid_constant__ LriGeom g, int r, const c128* __restrict__ evec,
                             c64* __restrict__ cR) {
  const long long per_k = (long long)g.NB * g.NBd, n = per_k * g.NK;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e / per_k);
    const int k3 = k % g.nk[2], k2 = (k / g.nk[2]) % g.nk[1], k1 = k / (g.nk[1] * g.nk[2]);
    const double ph = 2.0 * (((double)k1 / g.nk[0] + g.koff[0]) * g.R[r][0] +
                             ((double)k2 / g.nk[1] + g.koff[1]) * g.R[r][1] +
                             ((double)k3 / g.nk[2] + g.koff[2]) * g.R[r][2]);
    double sn, cs;
    sincospi(ph, &sn, &cs);
    const c128 v = evec[e];
    cR[e] = c64{(float)(cs * v.re - sn * v.im), (float)(cs * v.im + sn * v.re)};
  }
}

}  // namespace

template <>
void launch_lri_halfT<float>(const LriGeom& g, const double* ctil, const c128* evec, c64* T1, c64* /*T2*/,
                             cudaStream_t st) {
  const long long per_k = (long long)g.NB * g.NBd;
  long long amax = 0;
  for (int A = 0; A < g.n_atoms; ++A) amax = std::max(amax, (long long)g.atom_nx[A] * g.atom_nb[A] * g.NB);
  c64 *cR = nullptr, *At = nullptr;
  ::gw::g_alloc_count += 2;
  if (cudaMallocAsync(&cR, sizeof(c64) * per_k * g.NK, st) != cudaSuccess ||
      cudaMallocAsync(&At, sizeof(c64) * amax, st) != cudaSuccess) {
    // fall back to the direct kernel (same sums, FP64 arithmetic) when the staging does not fit
    cudaGetLastError();
    if (cR) cudaFreeAsync(cR, st);
    if (At) cudaFreeAsync(At, st);
    for (int A = 0; A < g.n_atoms; ++A) {
      long long total = (long long)g.NK * g.atom_nx[A] * g.atom_nb[A] * g.NBd;
      int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 64);
      ++::gw::g_launch_count, k_lri_halfT<float><<<blocks, 256, 0, st>>>(g, ctil, evec, T1, A);
    }
    return;
  }
  for (int r = 0; r < g.nR; ++r) {
    ++::gw::g_launch_count, k_phase_evec<<<(unsigned)std::min<long long>((per_k * g.NK + 255) / 256, 152LL * 32), 256,
                                           0, st>>>(g, r, evec, cR);
    for (int A = 0; A < g.n_atoms; ++A) {
      const int nx = g.atom_nx[A], nb = g.atom_nb[A];
      const long long rows = (long long)nx * nb;
      const double* cA = ctil + g.ctil_off[A] + (long long)r * rows * g.NB;
      ++::gw::g_launch_count, k_real_to_c64<<<(unsigned)std::min<long long>((rows * g.NB + 255) / 256, 152LL * 32), 256,
                                             0, st>>>(rows * g.NB, cA, At);
      launch_zgemm<float>((int)rows, g.NBd, g.NB, c64{1, 0}, At, g.NB, 0, OP_N, cR, g.NBd, per_k, OP_N,
                          c64{r == 0 ? 0.f : 1.f, 0}, T1 + g.t_off[A], g.NBd, rows * g.NBd, g.NK, st);
    }
  }
  cudaFreeAsync(cR, st);
  cudaFreeAsync(At, st);
}

// ---------------------------------------------------------------------------------------------
// M generation. One block per (row-k kk, block of MU ABFs); threads over (a, b) pairs.
// ---------------------------------------------------------------------------------------------
constexpr int MGEN_MU = 8;

__device__ __forceinline__ int aux_atom_of(const LriGeom& g, int mu) {
  int A = 0;
  while (A + 1 < g.n_atoms && mu >= g.atom_x0[A + 1]) ++A;
  return A;
}

template <typename T, typename Store>
__device__ __forceinline__ void mgen_body(const LriGeom& g, const cplx<T>* __restrict__ T1,
                                          const c128* __restrict__ evec, int q, int kk0, int mode, int a0, int na,
                                          int b0, int nb, Store store) {
  const int kk = blockIdx.x;
  int ktgt = g.ktab ? g.ktab[kk0 + kk] : kk0 + kk;
  int k3 = ktgt % g.nk[2], k2 = (ktgt / g.nk[2]) % g.nk[1], k1 = ktgt / (g.nk[1] * g.nk[2]);
  int q3 = q % g.nk[2], q2 = (q / g.nk[2]) % g.nk[1], q1 = q / (g.nk[1] * g.nk[2]);
  int kp;  // k' (b bands live here), k'+q (a bands live here)
  if (mode == MAP_K_IS_KK) {
    kp = ktgt;
  } else {
    kp = (((k1 - q1 + g.nk[0]) % g.nk[0]) * g.nk[1] + ((k2 - q2 + g.nk[1]) % g.nk[1])) * g.nk[2] +
         ((k3 - q3 + g.nk[2]) % g.nk[2]);
  }
  int p3 = kp % g.nk[2], p2 = (kp / g.nk[2]) % g.nk[1], p1 = kp / (g.nk[1] * g.nk[2]);
  int kpq = (((p1 + q1) % g.nk[0]) * g.nk[1] + ((p2 + q2) % g.nk[1])) * g.nk[2] + ((p3 + q3) % g.nk[2]);
  const c128* ck = evec + (long long)kp * g.NB * g.NBd;    // c(k')
  const c128* ckq = evec + (long long)kpq * g.NB * g.NBd;  // c(k'+q)
  const int mu_begin = blockIdx.y * MGEN_MU;
  const int mu_end = min(mu_begin + MGEN_MU, g.N);
  const int npair = na * nb;
  // (ABF, pair) flattened over the block's threads so that no lanes idle on a ragged pair count
  for (int idx = threadIdx.x; idx < (mu_end - mu_begin) * npair; idx += blockDim.x) {
    const int mu = mu_begin + idx / npair;
    const int p = idx % npair;
    const int A = aux_atom_of(g, mu);
    const int nbA = g.atom_nb[A], b0A = g.atom_b0[A];
    const int mul = mu - g.atom_x0[A];
    const cplx<T>* t1k = T1 + g.t_off[A] + (((long long)kp * g.atom_nx[A] + mul) * nbA) * g.NBd;
    const cplx<T>* t1kq = T1 + g.t_off[A] + (((long long)kpq * g.atom_nx[A] + mul) * nbA) * g.NBd;
    {
      const int a = a0 + p / nb, b = b0 + p % nb;
      T sr = 0, si = 0;
      for (int j = 0; j < nbA; ++j) {
        // c_{jb}(k') conj(T1^mu_{ja}(k'+q))
        c128 cjb = ck[(long long)(b0A + j) * g.NBd + b];
        cplx<T> t = t1kq[(long long)j * g.NBd + a];
        T cr = (T)cjb.re, ci = (T)cjb.im;
        sr += cr * t.re + ci * t.im;
        si += ci * t.re - cr * t.im;
        // conj(c_{ja}(k'+q)) T1^mu_{jb}(k')
        c128 cja = ckq[(long long)(b0A + j) * g.NBd + a];
        cplx<T> u = t1k[(long long)j * g.NBd + b];
        T dr = (T)cja.re, di = (T)cja.im;
        sr += dr * u.re + di * u.im;
        si += dr * u.im - di * u.re;
      }
      long long r = ((long long)kk * na + (p / nb)) * nb + (p % nb);
      store(r, mu, sr, si);
    }
  }
}

// Shared-memory form for fp32 (split-precision path). For one k' and a tile of MGT ABFs of one
// atom A (j, i run over the n_b(A) basis functions of A):
//   M^mu_{ab} = sum_j cK_{jb} conj(T1q^mu_{ja}) + sum_i conj(cQ_{ia}) T1k^mu_{ib}
//   cK = c(k')[A][b-range], cQ = c(k'+q)[A][a-range], T1q^mu = T1^mu(k'+q)[.][a-range], T1k^mu = T1^mu(k')[.][b-range]
// i.e. a complex product of K = 2 n_b(A) per ABF. The block (512 threads: one block of ~130 KB
// fits an SM, so the width buys the latency hiding) stages cK, cQ and the T1 slices of its ABFs
// in shared memory (fp32) once; threads run over (mu, a, b) outputs with the K loop in shared memory. Tiles never straddle atoms (tile t -> atom by the cumulative tile counts).
// Two thread mappings, picked per call shape by the plan's autotuner (both give bit-identical rows):
//   PAIR = false: one output (m, a, b) per thread, 512 threads;
//   PAIR = true:  one (a, b) pair per thread for all MGT ABFs of the tile (cK, cQ loaded once per
//                 j for MGT outputs), as many threads as pairs up to MGEN_SMEM_THREADS.
constexpr int MGT = 4;
constexpr int MGEN_SMEM_THREADS = 640;

__device__ __forceinline__ bool mgen_tile(const LriGeom& g, int t, int& A, int& mu0, int& cnt) {
  for (A = 0; A < g.n_atoms; ++A) {
    const int nt = (g.atom_nx[A] + MGT - 1) / MGT;
    if (t < nt) {
      mu0 = g.atom_x0[A] + t * MGT;
      cnt = min(MGT, g.atom_x0[A] + g.atom_nx[A] - mu0);
      return true;
    }
    t -= nt;
  }
  return false;
}

template <bool PAIR, typename Store>
__device__ __forceinline__ void mgen_smem_body(const LriGeom& g, const c64* __restrict__ T1,
                                               const c128* __restrict__ evec, int q, int kk0, int mode, int a0, int na,
                                               int b0, int nb, Store store) {
  extern __shared__ float2 sm2[];
  const int kk = blockIdx.x;
  int A, mu0, cnt;
  if (!mgen_tile(g, blockIdx.y, A, mu0, cnt)) return;
  int ktgt = g.ktab ? g.ktab[kk0 + kk] : kk0 + kk;
  int k3 = ktgt % g.nk[2], k2 = (ktgt / g.nk[2]) % g.nk[1], k1 = ktgt / (g.nk[1] * g.nk[2]);
  int q3 = q % g.nk[2], q2 = (q / g.nk[2]) % g.nk[1], q1 = q / (g.nk[1] * g.nk[2]);
  int kp;
  if (mode == MAP_K_IS_KK) {
    kp = ktgt;
  } else {
    kp = (((k1 - q1 + g.nk[0]) % g.nk[0]) * g.nk[1] + ((k2 - q2 + g.nk[1]) % g.nk[1])) * g.nk[2] +
         ((k3 - q3 + g.nk[2]) % g.nk[2]);
  }
  const int p3 = kp % g.nk[2], p2 = (kp / g.nk[2]) % g.nk[1], p1 = kp / (g.nk[1] * g.nk[2]);
  const int kpq = (((p1 + q1) % g.nk[0]) * g.nk[1] + ((p2 + q2) % g.nk[1])) * g.nk[2] + ((p3 + q3) % g.nk[2]);
  const int nbA = g.atom_nb[A], b0A = g.atom_b0[A];
  // shared layout (float2): cK [nbA][nb], cQ [nbA][na], T1q [MGT][nbA][na], T1k [MGT][nbA][nb]
  float2* cK = sm2;
  float2* cQ = cK + nbA * nb;
  float2* tq = cQ + nbA * na;
  float2* tk = tq + MGT * nbA * na;
  const c128* ck = evec + (long long)kp * g.NB * g.NBd;
  const c128* ckq = evec + (long long)kpq * g.NB * g.NBd;
  for (int e = threadIdx.x; e < nbA * nb; e += blockDim.x) {
    const c128 v = ck[(long long)(b0A + e / nb) * g.NBd + b0 + e % nb];
    cK[e] = make_float2((float)v.re, (float)v.im);
  }
  for (int e = threadIdx.x; e < nbA * na; e += blockDim.x) {
    const c128 v = ckq[(long long)(b0A + e / na) * g.NBd + a0 + e % na];
    cQ[e] = make_float2((float)v.re, (float)v.im);
  }
  for (int e = threadIdx.x; e < cnt * nbA * na; e += blockDim.x) {
    const int m = e / (nbA * na), rest = e % (nbA * na), j = rest / na, a = rest % na;
    const c64 v = T1[g.t_off[A] + (((long long)kpq * g.atom_nx[A] + (mu0 - g.atom_x0[A] + m)) * nbA + j) * g.NBd + a0 + a];
    tq[e] = make_float2(v.re, v.im);
  }
  for (int e = threadIdx.x; e < cnt * nbA * nb; e += blockDim.x) {
    const int m = e / (nbA * nb), rest = e % (nbA * nb), j = rest / nb, b = rest % nb;
    const c64 v = T1[g.t_off[A] + (((long long)kp * g.atom_nx[A] + (mu0 - g.atom_x0[A] + m)) * nbA + j) * g.NBd + b0 + b];
    tk[e] = make_float2(v.re, v.im);
  }
  __syncthreads();
  const int npair = na * nb;
  if constexpr (PAIR) {
    for (int pr = threadIdx.x; pr < npair; pr += blockDim.x) {
      const int a = pr / nb, b = pr % nb;
      float sr[MGT], si[MGT];
#pragma unroll
      for (int m = 0; m < MGT; ++m) sr[m] = si[m] = 0.f;
      for (int j = 0; j < nbA; ++j) {
        const float2 c = cK[j * nb + b], d = cQ[j * na + a];
#pragma unroll
        for (int m = 0; m < MGT; ++m) {
          if (m < cnt) {
            const float2 t = tq[(m * nbA + j) * na + a], u = tk[(m * nbA + j) * nb + b];
            sr[m] = fmaf(c.x, t.x, fmaf(c.y, t.y, sr[m]));     // c conj(t)
            si[m] = fmaf(c.y, t.x, fmaf(-c.x, t.y, si[m]));
            sr[m] = fmaf(d.x, u.x, fmaf(d.y, u.y, sr[m]));     // conj(d) u
            si[m] = fmaf(d.x, u.y, fmaf(-d.y, u.x, si[m]));
          }
        }
      }
#pragma unroll
      for (int m = 0; m < MGT; ++m)
        if (m < cnt) store(((long long)kk * na + a) * nb + b, mu0 + m, sr[m], si[m]);
    }
  } else {
    for (int idx = threadIdx.x; idx < cnt * npair; idx += blockDim.x) {
      const int m = idx / npair, pr = idx % npair, a = pr / nb, b = pr % nb;
      const float2* tqm = tq + m * nbA * na;
      const float2* tkm = tk + m * nbA * nb;
      float sr = 0.f, si = 0.f;
      for (int j = 0; j < nbA; ++j) {
        const float2 c = cK[j * nb + b], t = tqm[j * na + a];     // c conj(t)
        sr = fmaf(c.x, t.x, fmaf(c.y, t.y, sr));
        si = fmaf(c.y, t.x, fmaf(-c.x, t.y, si));
        const float2 d = cQ[j * na + a], u = tkm[j * nb + b];     // conj(d) u
        sr = fmaf(d.x, u.x, fmaf(d.y, u.y, sr));
        si = fmaf(d.x, u.y, fmaf(-d.y, u.x, si));
      }
      store(((long long)kk * na + a) * nb + b, mu0 + m, sr, si);
    }
  }
}

int mgen_tiles(const LriGeom& g) {
  int t = 0;
  for (int A = 0; A < g.n_atoms; ++A) t += (g.atom_nx[A] + MGT - 1) / MGT;
  return t;
}

// threads per block of the shared-memory M kernels
int mgen_threads(bool pair, int na, int nb) {
  if (!pair) return 512;
  const int n = ((na * nb + 31) / 32) * 32;
  return std::max(64, std::min(MGEN_SMEM_THREADS, n));
}

size_t mgen_smem(const LriGeom& g, int na, int nb) {
  int nbA = 0;
  for (int A = 0; A < g.n_atoms; ++A) nbA = std::max(nbA, g.atom_nb[A]);
  return sizeof(float2) * (size_t)nbA * (na + nb) * (1 + MGT);
}

template <bool PAIR>
__global__ void __launch_bounds__(MGEN_SMEM_THREADS) k_mgen_smem(const __grid_constant__ LriGeom g, const c64* __restrict__ T1, const c128* __restrict__ evec, int q, int kk0, int mode, int a0,
                            int na, int b0, int nb, c64* __restrict__ out, long long s_r, long long s_mu) {
  mgen_smem_body<PAIR>(g, T1, evec, q, kk0, mode, a0, na, b0, nb, [&](long long r, int mu, float re, float im) {
    out[r * s_r + (long long)mu * s_mu] = c64{re, im};
  });
}

template <typename T>
__global__ void k_mgen(const __grid_constant__ LriGeom g, const cplx<T>* __restrict__ T1, const c128* __restrict__ evec, int q, int kk0, int mode,
                       int a0, int na, int b0, int nb, cplx<T>* __restrict__ out, long long s_r, long long s_mu) {
  mgen_body<T>(g, T1, evec, q, kk0, mode, a0, na, b0, nb, [&](long long r, int mu, T re, T im) {
    out[r * s_r + (long long)mu * s_mu] = cplx<T>{re, im};
  });
}

template <typename T>
void launch_mgen(const LriGeom& g, const cplx<T>* T1, const cplx<T>* /*T2*/, const c128* evec, int q, int kk0,
                 int nkk, MapMode mode, int a0, int na, int b0, int nb, cplx<T>* out, long long s_r, long long s_mu,
                 cudaStream_t st, int /*variant*/) {
  dim3 grid(nkk, (g.N + MGEN_MU - 1) / MGEN_MU);
  ++::gw::g_launch_count, k_mgen<T><<<grid, 256, 0, st>>>(g, T1, evec, q, kk0, (int)mode, a0, na, b0, nb, out, s_r, s_mu);
}
template void launch_mgen<double>(const LriGeom&, const c128*, const c128*, const c128*, int, int, int, MapMode, int,
                                  int, int, int, c128*, long long, long long, cudaStream_t, int);

// fp32: the shared-memory kernel when its staging fits, else the plain one
template <>
void launch_mgen<float>(const LriGeom& g, const c64* T1, const c64* T2, const c128* evec, int q, int kk0, int nkk,
                        MapMode mode, int a0, int na, int b0, int nb, c64* out, long long s_r, long long s_mu,
                        cudaStream_t st, int variant) {
  const size_t sm = mgen_smem(g, na, nb);
  if (sm > 200 * 1024) {
    dim3 grid(nkk, (g.N + MGEN_MU - 1) / MGEN_MU);
    ++::gw::g_launch_count, k_mgen<float><<<grid, 256, 0, st>>>(g, T1, evec, q, kk0, (int)mode, a0, na, b0, nb, out, s_r,
                                                                s_mu);
    return;
  }
  (void)T2;
  dim3 grid(nkk, mgen_tiles(g));
  const int nt = mgen_threads(variant != 0, na, nb);
  if (variant) {
    cudaFuncSetAttribute(k_mgen_smem<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    ++::gw::g_launch_count, k_mgen_smem<true><<<grid, nt, sm, st>>>(g, T1, evec, q, kk0, (int)mode, a0, na, b0, nb, out,
                                                                    s_r, s_mu);
  } else {
    cudaFuncSetAttribute(k_mgen_smem<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    ++::gw::g_launch_count, k_mgen_smem<false><<<grid, nt, sm, st>>>(g, T1, evec, q, kk0, (int)mode, a0, na, b0, nb, out,
                                                                     s_r, s_mu);
  }
}

// Sigma_c rows, streamed (split-precision path). a_r(mu) = C^mu_{ab}(k, k - q) = M^mu_{ab}(k', q),
// k' = k - q, a in the Sigma window (na <= SIG_NA, bands at k), b over the nb bands at k':
//   M^mu_{ab} = sum_j c_{jb}(k') conj(T1^mu_{ja}(k)) + sum_i conj(c_{ia}(k)) T1^mu_{ib}(k'),
// i, j over the n_b(A) basis functions of mu's atom A. The large operand is the slab
// T1^mu(k')[i][b] (n_b(A) x nb per ABF): each thread owns one b and SIG_G ABFs of the block's
// tile, reads the slabs once (coalesced along b) and the eigenvector c(k')[i][b] once for all of
// them; the small pieces (T1^mu(k)[j][a] and c(k)[i][a] over the window) sit in shared memory.
// The rows are HBM streams of arithmetic intensity ~4 flop/byte, so this is CUDA-core work.
constexpr int SIG_NA = 8;   // largest Sigma window of this kernel
constexpr int SIG_G = 4;    // ABFs per block
constexpr int SIG_AT = 4;   // window bands per thread: the block's threads split the window in halves

__global__ void __launch_bounds__(256, 3) k_mgen_sig(const __grid_constant__ LriGeom g, const c64* __restrict__ T1,
                                                  const c128* __restrict__ evec, int q, int kk0, int a0, int na,
                                                  int nb, c64* __restrict__ out, long long s_r, long long s_mu) {
  __shared__ float2 sQ[SIG_G][48][SIG_NA];   // T1^mu(k)[j][a] (n_b(A) <= 48)
  __shared__ float2 sC[48][SIG_NA];          // c(k)[i][a]
  const int kk = blockIdx.x;
  int t = blockIdx.y, A = 0;
  for (; A < g.n_atoms; ++A) {
    const int nt = (g.atom_nx[A] + SIG_G - 1) / SIG_G;
    if (t < nt) break;
    t -= nt;
  }
  if (A >= g.n_atoms) return;
  const int mu0 = g.atom_x0[A] + t * SIG_G, cnt = min(SIG_G, g.atom_x0[A] + g.atom_nx[A] - mu0);
  const int ktgt = g.ktab ? g.ktab[kk0 + kk] : kk0 + kk;
  const int k3 = ktgt % g.nk[2], k2 = (ktgt / g.nk[2]) % g.nk[1], k1 = ktgt / (g.nk[1] * g.nk[2]);
  const int q3 = q % g.nk[2], q2 = (q / g.nk[2]) % g.nk[1], q1 = q / (g.nk[1] * g.nk[2]);
  const int kp = (((k1 - q1 + g.nk[0]) % g.nk[0]) * g.nk[1] + ((k2 - q2 + g.nk[1]) % g.nk[1])) * g.nk[2] +
                 ((k3 - q3 + g.nk[2]) % g.nk[2]);
  const int nbA = g.atom_nb[A], b0A = g.atom_b0[A], nxA = g.atom_nx[A];
  const c128* ck = evec + (long long)kp * g.NB * g.NBd;     // c(k')
  const c128* cq = evec + (long long)ktgt * g.NB * g.NBd;   // c(k)
  for (int e = threadIdx.x; e < nbA * SIG_NA; e += blockDim.x) {
    const int i = e / SIG_NA, a = e % SIG_NA;
    float2 v = make_float2(0.f, 0.f);
    if (a < na) {
      const c128 c = cq[(long long)(b0A + i) * g.NBd + a0 + a];
      v = make_float2((float)c.re, (float)c.im);
    }
    sC[i][a] = v;
  }
  for (int e = threadIdx.x; e < SIG_G * nbA * SIG_NA; e += blockDim.x) {
    const int m = e / (nbA * SIG_NA), rest = e % (nbA * SIG_NA), j = rest / SIG_NA, a = rest % SIG_NA;
    float2 v = make_float2(0.f, 0.f);
    if (m < cnt && a < na) {
      const c64 x = T1[g.t_off[A] + (((long long)ktgt * nxA + (mu0 - g.atom_x0[A] + m)) * nbA + j) * g.NBd + a0 + a];
      v = make_float2(x.re, x.im);
    }
    sQ[m][j][a] = v;
  }
  __syncthreads();
  const c64* U = T1 + g.t_off[A] + ((long long)kp * nxA + (mu0 - g.atom_x0[A])) * nbA * g.NBd;
  const long long us = (long long)nbA * g.NBd;     // between the slabs of consecutive ABFs
  // thread = (window half, band b): each warp covers 32 consecutive b of one half
  const int nhalf = (na + SIG_AT - 1) / SIG_AT;
  const int nbt = blockDim.x / nhalf;
  const int ah = threadIdx.x / nbt, ab0 = SIG_AT * ah;
  for (int b = threadIdx.x % nbt; b < nb && ah < nhalf; b += nbt) {
    float ar[SIG_G][SIG_AT], ai[SIG_G][SIG_AT];
#pragma unroll
    for (int m = 0; m < SIG_G; ++m)
#pragma unroll
      for (int a = 0; a < SIG_AT; ++a) ar[m][a] = ai[m][a] = 0.f;
    for (int i = 0; i < nbA; ++i) {
      const c128 cb = ck[(long long)(b0A + i) * g.NBd + b];
      const float cr = (float)cb.re, ci = (float)cb.im;
      float ur[SIG_G], ui[SIG_G];
#pragma unroll
      for (int m = 0; m < SIG_G; ++m) {
        const c64 u = (m < cnt) ? U[m * us + (long long)i * g.NBd + b] : c64{0.f, 0.f};
        ur[m] = u.re;
        ui[m] = u.im;
      }
#pragma unroll
      for (int a = 0; a < SIG_AT; ++a) {
        const float2 d = sC[i][ab0 + a];
#pragma unroll
        for (int m = 0; m < SIG_G; ++m) {
          const float2 tq = sQ[m][i][ab0 + a];
          // c_{ib}(k') conj(T1^mu_{ia}(k)) + conj(c_{ia}(k)) T1^mu_{ib}(k')
          ar[m][a] = fmaf(cr, tq.x, fmaf(ci, tq.y, fmaf(d.x, ur[m], fmaf(d.y, ui[m], ar[m][a]))));
          ai[m][a] = fmaf(ci, tq.x, fmaf(-cr, tq.y, fmaf(d.x, ui[m], fmaf(-d.y, ur[m], ai[m][a]))));
        }
      }
    }
#pragma unroll
    for (int a = 0; a < SIG_AT; ++a) {
      if (ab0 + a >= na) continue;
      const long long r = ((long long)kk * na + ab0 + a) * nb + b;
#pragma unroll
      for (int m = 0; m < SIG_G; ++m)
        if (m < cnt) out[r * s_r + (long long)(mu0 + m) * s_mu] = c64{ar[m][a], ai[m][a]};
    }
  }
}

bool launch_mgen_sig(const LriGeom& g, const c64* T1, const c128* evec, int q, int kk0, int nkk, int a0, int na,
                     int nb, c64* out, long long s_r, long long s_mu, cudaStream_t st) {
  if (na > SIG_NA) return false;
  for (int A = 0; A < g.n_atoms; ++A)
    if (g.atom_nb[A] > 48) return false;
  int tiles = 0;
  for (int A = 0; A < g.n_atoms; ++A) tiles += (g.atom_nx[A] + SIG_G - 1) / SIG_G;
  dim3 grid(nkk, tiles);
  // one thread per (window half, band b); whole warps per half, at most 128 threads per half
  const int nhalf = (na + SIG_AT - 1) / SIG_AT;
  const int nt = nhalf * std::min(128, (nb + 31) / 32 * 32);
  ++::gw::g_launch_count, k_mgen_sig<<<grid, nt, 0, st>>>(g, T1, evec, q, kk0, a0, na, nb, out, s_r, s_mu);
  return true;
}

// chi0 pair rows, streamed (split-precision path): M^mu_{ab}(k, q) for a over na unoccupied bands
// at k + q (the wide side) and b over nb <= CHI_NB occupied bands at k,
//   M^mu_{ab} = sum_j c_{jb}(k) conj(T1^mu_{ja}(k + q)) + sum_i conj(c_{ia}(k + q)) T1^mu_{ib}(k),
// written as the fp32 plane raw[mu][kofs + 2 r + {0, 1}], r = (kk * na + a) * nb + b, with the
// largest |re|, |im| into absmax. Each thread owns one a and SIG_G ABFs: the slabs
// T1^mu(k + q)[j][a] and c(k + q)[i][a] are read once along a; T1^mu(k)[i][b] and c(k)[j][b] sit
// in shared memory. CHI_NB (4 or 8) bounds the occupied bands of one launch; the FMA work and the
// accumulator registers scale with it.
template <int CHI_NB>
__global__ void __launch_bounds__(128) k_mgen_chi(const __grid_constant__ LriGeom g, const c64* __restrict__ T1,
                                                  const c128* __restrict__ evec, int q, int kk0, int a0, int na,
                                                  int b0, int nb, float* __restrict__ raw, long long ldk,
                                                  long long kofs, unsigned* __restrict__ absmax) {
  __shared__ float2 sT[SIG_G][48][CHI_NB];   // T1^mu(k)[i][b]
  __shared__ float2 sC[48][CHI_NB];          // c(k)[j][b]
  const int kk = blockIdx.x;
  int t = blockIdx.y, A = 0;
  for (; A < g.n_atoms; ++A) {
    const int nt = (g.atom_nx[A] + SIG_G - 1) / SIG_G;
    if (t < nt) break;
    t -= nt;
  }
  float amax = 0.f;
  if (A < g.n_atoms) {
    const int mu0 = g.atom_x0[A] + t * SIG_G, cnt = min(SIG_G, g.atom_x0[A] + g.atom_nx[A] - mu0);
    const int k = g.ktab ? g.ktab[kk0 + kk] : kk0 + kk;
    const int k3 = k % g.nk[2], k2 = (k / g.nk[2]) % g.nk[1], k1 = k / (g.nk[1] * g.nk[2]);
    const int q3 = q % g.nk[2], q2 = (q / g.nk[2]) % g.nk[1], q1 = q / (g.nk[1] * g.nk[2]);
    const int kq = (((k1 + q1) % g.nk[0]) * g.nk[1] + ((k2 + q2) % g.nk[1])) * g.nk[2] + ((k3 + q3) % g.nk[2]);
    const int nbA = g.atom_nb[A], b0A = g.atom_b0[A], nxA = g.atom_nx[A];
    const c128* ck = evec + (long long)k * g.NB * g.NBd;
    const c128* ckq = evec + (long long)kq * g.NB * g.NBd;
    for (int e = threadIdx.x; e < nbA * CHI_NB; e += blockDim.x) {
      const int j = e / CHI_NB, b = e % CHI_NB;
      float2 v = make_float2(0.f, 0.f);
      if (b < nb) {
        const c128 c = ck[(long long)(b0A + j) * g.NBd + b0 + b];
        v = make_float2((float)c.re, (float)c.im);
      }
      sC[j][b] = v;
    }
    for (int e = threadIdx.x; e < SIG_G * nbA * CHI_NB; e += blockDim.x) {
      const int m = e / (nbA * CHI_NB), rest = e % (nbA * CHI_NB), i = rest / CHI_NB, b = rest % CHI_NB;
      float2 v = make_float2(0.f, 0.f);
      if (m < cnt && b < nb) {
        const c64 x = T1[g.t_off[A] + (((long long)k * nxA + (mu0 - g.atom_x0[A] + m)) * nbA + i) * g.NBd + b0 + b];
        v = make_float2(x.re, x.im);
      }
      sT[m][i][b] = v;
    }
    __syncthreads();
    const c64* U = T1 + g.t_off[A] + ((long long)kq * nxA + (mu0 - g.atom_x0[A])) * nbA * g.NBd;
    const long long us = (long long)nbA * g.NBd;
    for (int a = threadIdx.x; a < na; a += blockDim.x) {
      float ar[SIG_G][CHI_NB], ai[SIG_G][CHI_NB];
#pragma unroll
      for (int m = 0; m < SIG_G; ++m)
#pragma unroll
        for (int b = 0; b < CHI_NB; ++b) ar[m][b] = ai[m][b] = 0.f;
      for (int j = 0; j < nbA; ++j) {
        const c128 ca = ckq[(long long)(b0A + j) * g.NBd + a0 + a];   // c_{ja}(k + q)
        const float dr = (float)ca.re, di = (float)ca.im;
        float ur[SIG_G], ui[SIG_G];
#pragma unroll
        for (int m = 0; m < SIG_G; ++m) {
          const c64 u = (m < cnt) ? U[m * us + (long long)j * g.NBd + a0 + a] : c64{0.f, 0.f};   // T1^mu_{ja}(k+q)
          ur[m] = u.re;
          ui[m] = u.im;
        }
#pragma unroll
        for (int b = 0; b < CHI_NB; ++b) {
          const float2 c = sC[j][b];
#pragma unroll
          for (int m = 0; m < SIG_G; ++m) {
            const float2 tk = sT[m][j][b];
            // c_{jb}(k) conj(T1^mu_{ja}(k+q)) + conj(c_{ja}(k+q)) T1^mu_{jb}(k)
            ar[m][b] = fmaf(c.x, ur[m], fmaf(c.y, ui[m], fmaf(dr, tk.x, fmaf(di, tk.y, ar[m][b]))));
            ai[m][b] = fmaf(c.y, ur[m], fmaf(-c.x, ui[m], fmaf(dr, tk.y, fmaf(-di, tk.x, ai[m][b]))));
          }
        }
      }
#pragma unroll
      for (int m = 0; m < SIG_G; ++m) {
        if (m >= cnt) continue;
        float* row = raw + (long long)(mu0 + m) * ldk + kofs + 2 * (((long long)kk * na + a) * nb);
#pragma unroll
        for (int b = 0; b < CHI_NB; ++b) {
          if (b >= nb) continue;
          *reinterpret_cast<float2*>(row + 2 * b) = make_float2(ar[m][b], ai[m][b]);
          amax = fmaxf(amax, fmaxf(fabsf(ar[m][b]), fabsf(ai[m][b])));
        }
      }
    }
  }
  if (absmax) {
    // every thread gets here (whole warps); non-negative floats order like their bit patterns
    const unsigned mm = __reduce_max_sync(0xffffffffu, __float_as_uint(amax));
    if ((threadIdx.x & 31) == 0) atomicMax(absmax, mm);
  }
}

bool launch_mgen_chi(const LriGeom& g, const c64* T1, const c128* evec, int q, int kk0, int nkk, int a0, int na,
                     int b0, int nb, float* raw, long long ldk, long long kofs, unsigned* absmax, cudaStream_t st) {
  if (nb > 8) return false;
  for (int A = 0; A < g.n_atoms; ++A)
    if (g.atom_nb[A] > 48) return false;
  int tiles = 0;
  for (int A = 0; A < g.n_atoms; ++A) tiles += (g.atom_nx[A] + SIG_G - 1) / SIG_G;
  dim3 grid(nkk, tiles);
  // one thread per unoccupied band (whole warps, at most 128)
  const int nt = std::min(128, (na + 31) / 32 * 32);
  if (nb <= 4)
    ++::gw::g_launch_count, k_mgen_chi<4><<<grid, nt, 0, st>>>(g, T1, evec, q, kk0, a0, na, b0, nb, raw, ldk, kofs, absmax);
  else
    ++::gw::g_launch_count, k_mgen_chi<8><<<grid, nt, 0, st>>>(g, T1, evec, q, kk0, a0, na, b0, nb, raw, ldk, kofs, absmax);
  return true;
}

// Operand planes for the tensor-core chi0 (row mu, K index kofs + 2r + {0, 1}):
//   raw:  fp32 (re, im) of M^mu_r -- read by the transform warps that build the weighted A side;
//   B1 pieces: split of (re, im);  B2 pieces: split of (-im, re)  (the complex product's second
//   half, so that one K-concatenated MMA over [B1; B2] yields Re and Im columns).
// BF16: three pieces h = bf16(x), m = bf16(x - h), l = bf16(x - h - m).
// TF32: two pieces h = x rounded to 10 explicit mantissa bits (fp32 container), l = x - h.
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7f800000u) == 0x7f800000u) return x;          // inf / nan unchanged
  u += 0x1000u;                                             // round half away on the 13 dropped bits
  u &= 0xffffe000u;
  return __uint_as_float(u);
}

struct PlanePtrs {
  float* raw;
  void* b[6];      // B1 pieces then B2 pieces (b[0] NULL: raw plane only)
  unsigned* absmax;
};

template <bool SMEM, bool PAIR>
__global__ void __launch_bounds__(MGEN_SMEM_THREADS) k_mgen_planes(const __grid_constant__ LriGeom g, const c64* __restrict__ T1, const c128* __restrict__ evec, int q, int kk0, int a0,
                              int na, int b0, int nb, PlanePtrs P, long long ldk, long long kofs, int tf32) {
  float amax = 0.f;
  auto st = [&](long long r, int mu, float re, float im) {
    const long long e = (long long)mu * ldk + kofs + 2 * r;
    *reinterpret_cast<float2*>(P.raw + e) = make_float2(re, im);
    amax = fmaxf(amax, fmaxf(fabsf(re), fabsf(im)));
    if (!P.b[0]) return;
    const float v1[2] = {re, im}, v2[2] = {-im, re};
    if (tf32) {
      for (int half = 0; half < 2; ++half) {
        const float* v = half ? v2 : v1;
        const float h0 = tf32_round(v[0]), h1 = tf32_round(v[1]);
        *reinterpret_cast<float2*>(reinterpret_cast<float*>(P.b[2 * half + 0]) + e) = make_float2(h0, h1);
        *reinterpret_cast<float2*>(reinterpret_cast<float*>(P.b[2 * half + 1]) + e) =
            make_float2(v[0] - h0, v[1] - h1);
      }
    } else {
      for (int half = 0; half < 2; ++half) {
        const float* v = half ? v2 : v1;
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[0], v[1]);
        const float2 hf = __bfloat1622float2(h);
        const float r0 = v[0] - hf.x, r1 = v[1] - hf.y;
        const __nv_bfloat162 m = __floats2bfloat162_rn(r0, r1);
        const float2 mf = __bfloat1622float2(m);
        const __nv_bfloat162 l = __floats2bfloat162_rn(r0 - mf.x, r1 - mf.y);
        *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(P.b[3 * half + 0]) + e) = h;
        *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(P.b[3 * half + 1]) + e) = m;
        *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(P.b[3 * half + 2]) + e) = l;
      }
    }
  };
  if constexpr (SMEM)
    mgen_smem_body<PAIR>(g, T1, evec, q, kk0, MAP_K_IS_KK, a0, na, b0, nb, st);
  else
    mgen_body<float>(g, T1, evec, q, kk0, MAP_K_IS_KK, a0, na, b0, nb, st);
  if (P.absmax) {
    // every thread of the block gets here (block sizes are multiples of 32); non-negative
    // floats order like their bit patterns
    const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(amax));
    if ((threadIdx.x & 31) == 0) atomicMax(P.absmax, m);
  }
}

void launch_mgen_planes(const LriGeom& g, const c64* T1, const c128* evec, int q, int kk0, int nkk, int a0, int na,
                        int b0, int nb, float* raw, void* const* bplanes, long long ldk, long long kofs, int tf32,
                        cudaStream_t st, int variant, unsigned* absmax) {
  PlanePtrs P{};
  P.raw = raw;
  P.absmax = absmax;
  if (bplanes)
    for (int i = 0; i < (tf32 ? 4 : 6); ++i) P.b[i] = bplanes[i];
  const size_t sm = mgen_smem(g, na, nb);
  if (sm <= 200 * 1024) {
    dim3 grid(nkk, mgen_tiles(g));
    const int nt = mgen_threads(variant != 0, na, nb);
    if (variant) {
      cudaFuncSetAttribute(k_mgen_planes<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      ++::gw::g_launch_count, k_mgen_planes<true, true><<<grid, nt, sm, st>>>(g, T1, evec, q, kk0, a0, na, b0, nb, P, ldk,
                                                                              kofs, tf32);
    } else {
      cudaFuncSetAttribute(k_mgen_planes<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      ++::gw::g_launch_count, k_mgen_planes<true, false><<<grid, nt, sm, st>>>(g, T1, evec, q, kk0, a0, na, b0, nb, P, ldk,
                                                                               kofs, tf32);
    }
  } else {
    dim3 grid(nkk, (g.N + MGEN_MU - 1) / MGEN_MU);
    ++::gw::g_launch_count, k_mgen_planes<false, false><<<grid, 256, 0, st>>>(g, T1, evec, q, kk0, a0, na, b0, nb, P, ldk,
                                                                               kofs, tf32);
  }
}

}  // namespace gw
