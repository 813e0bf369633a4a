// Internal declarations shared by the CUDA translation units of libgw.
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>

#include "../../include/gw.h"

namespace gw {

// number of kernels this library has launched (process-wide, host side)
extern std::atomic<unsigned long long> g_launch_count;
extern std::atomic<unsigned long long> g_alloc_count;   // device allocations (cudaMalloc) made by the library

// complex helpers (device and host)
template <typename T> struct cplx { T re, im; };
using c64 = cplx<float>;
using c128 = cplx<double>;

template <typename T> __host__ __device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T> __host__ __device__ __forceinline__ cplx<T> cmulc(cplx<T> a, cplx<T> b) {  // a * conj(b)
  return {a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im};
}
template <typename T> __host__ __device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) {
  return {a.re + b.re, a.im + b.im};
}
template <typename T> __host__ __device__ __forceinline__ cplx<T> cfma(cplx<T> a, cplx<T> b, cplx<T> c) {  // a*b + c
  return {fma(a.re, b.re, fma(-a.im, b.im, c.re)), fma(a.re, b.im, fma(a.im, b.re, c.im))};
}
template <typename T> __host__ __device__ __forceinline__ cplx<T> cconj(cplx<T> a) { return {a.re, -a.im}; }

// device status word bits (written by kernels, read by the host after a call)
enum : int {
  ST_NOT_PD = 1,     // non-positive Cholesky pivot
  ST_TIMEOUT = 2,    // a bounded wait gave up
  ST_BADARG = 4,     // kernel-side bounds check tripped
  ST_NOCONV = 8      // an iteration did not converge (informational)
};

// operand modes of the generic complex GEMM
enum Op { OP_N = 0, OP_T = 1, OP_C = 2, OP_CONJ = 3 };   // as is, transpose, conj-transpose, conj only

// ---- kernels (launch wrappers), grouped by translation unit ---------------------------------

// k_lri.cu -- step (a)
// T1_A[k][mu][i][b] = sum_R e^{2 pi i k.R} sum_j C~_A[R][mu][i][j] c[k][j][b]              (mu, i on A)
// T2_A[k][mu][j][a] = sum_R e^{-2 pi i k.R} sum_i C~_A[R][mu][j][i] conj(c[k][i][a])      (mu, j on A)
struct LriGeom {
  int n_atoms, NK, NB, NBd, N, nR;
  int nk[3];
  double koff[3];              // shift of the k mesh (fractional); the q mesh is not shifted
  const int* ktab;             // device: target k of row block kk0 + kk (NULL: k = kk0 + kk)
  int atom_b0[64], atom_nb[64], atom_x0[64], atom_nx[64];
  long long ctil_off[64];      // element offset of atom block in ctil_R
  long long t_off[64];         // element offset of atom block in T1/T2
  int R[64][3];
};
template <typename T>
void launch_lri_halfT(const LriGeom& g, const double* ctil, const c128* evec, cplx<T>* T1, cplx<T>* T2,
                      cudaStream_t st);

// M^mu_{ab}(k', q) for a in [a0, a0+na) at k'+q and b in [b0, b0+nb) at k', for the k' of each row block.
// Row index r = ((kk * na) + a) * nb + b for kk in [0, nkk); k' = kmap(kk) (see MapMode).
// out element (r, mu) at out[r * s_r + mu * s_mu].
// variant (fp32 shared-memory kernels): thread mapping, 0 = one output per thread, 1 = one (a, b)
// pair per thread over the tile's ABFs; both give bit-identical rows (picked by MgenTuner).
enum MapMode { MAP_K_IS_KK = 0, MAP_K_IS_KK_MINUS_Q = 1 };
template <typename T>
void launch_mgen(const LriGeom& g, const cplx<T>* T1, const cplx<T>* T2, const c128* evec, int q,
                 int kk0, int nkk, MapMode mode, int a0, int na, int b0, int nb, cplx<T>* out, long long s_r,
                 long long s_mu, cudaStream_t st, int variant = 0);
// Sigma_c rows of the split path, streamed (window of at most 8 bands, n_b(A) <= 48); returns
// false when the shape is outside that range (the caller then uses launch_mgen<float>)
bool launch_mgen_sig(const LriGeom& g, const c64* T1, const c128* evec, int q, int kk0, int nkk, int a0, int na,
                     int nb, c64* out, long long s_r, long long s_mu, cudaStream_t st);
// chi0 pair rows of the split path as the fp32 plane (streamed; at most 8 occupied bands,
// n_b(A) <= 48), largest |re|, |im| into absmax; false outside that range
bool launch_mgen_chi(const LriGeom& g, const c64* T1, const c128* evec, int q, int kk0, int nkk, int a0, int na,
                     int b0, int nb, float* raw, long long ldk, long long kofs, unsigned* absmax, cudaStream_t st);
// split planes for the tensor-core chi0 B operand: for row mu, K index 2r + {0: re, 1: im}
// raw fp32 plane + B1/B2 split planes (3 BF16 pieces or 2 TF32 pieces each), see k_lri.cu
// bplanes may be NULL (raw plane only); absmax (may be NULL) receives max |re|, |im| of the rows
// written, as float bits (atomicMax; the caller zeroes it)
void launch_mgen_planes(const LriGeom& g, const c64* T1, const c128* evec, int q, int kk0, int nkk, int a0, int na,
                        int b0, int nb, float* raw, void* const* bplanes, long long ldk, long long kofs, int tf32,
                        cudaStream_t st, int variant = 0, unsigned* absmax = nullptr);

// k_linalg.cu
template <typename T>
void launch_zgemm(int m, int n, int k, cplx<T> alpha, const cplx<T>* A, long long lda, long long sA, Op opA,
                  const cplx<T>* B, long long ldb, long long sB, Op opB, cplx<T> beta, cplx<T>* C,
                  long long ldc, long long sC, int batch, cudaStream_t st);
// chi0[w][mu][nu] += scale * sum_r w_w(D_r) Mt[mu][r] conj(Mt[nu][r]),  Mt row-major [N][ldm]
template <typename T>
void launch_chi0_simt(int N, int K, const cplx<T>* Mt, long long ldm, const float* delta_f, const double* delta_d,
                      const double* freq, int nw, double scale, c128* chi0, cudaStream_t st);
// per matrix b: A[b] (Hermitian PD, row-major N x N, FP64) -> A[b] := A[b]^{-1} - I. Sets ST_NOT_PD.
void launch_chol_inv_minus_I(int N, c128* A, int batch, long long stride, c128* work, int* status,
                             cudaStream_t st);
template <typename T> void launch_axpby_identity(int N, cplx<T>* A, long long s, int batch, T diag, cudaStream_t st);
void launch_take_both(int N, const c128* C, long long s, int batch, float d, c64* X, c64* XH, cudaStream_t st);
void launch_dev_identity(int N, const c64* T, long long total, unsigned* dev, cudaStream_t st);
void launch_convert(int n, const c128* in, c64* out, cudaStream_t st);
// dominant eigenpair of a Hermitian matrix by power iteration (FP64)
void launch_power_iter(int N, const c128* A, c128* x, double* lam, int iters, cudaStream_t st);
// A += alpha * x x^H
void launch_rank1(int N, c128* A, const c128* x, double alpha, cudaStream_t st);
// q=0 head and wing vector: head[w], h[w][nu]
template <typename T>
void launch_head_wings(int N, int K, const cplx<T>* Mt, long long ldm, const double* delta, const c128* pq,
                       const double* freq, int nw, double head_pref, double* head, c128* h, cudaStream_t st);
// direction-averaged q = 0 (head_wings = 2): Cartesian head tensor A6[w][6] and wings h3[w][3][N]
// (accumulated); the moments of the Schur complement over the direction rule; the rank-4 update
template <typename T>
void launch_head_wings3(int N, int K, const cplx<T>* Mt, long long ldm, const double* delta, const c128* pq3,
                        long long ldp, const double* freq, int nw, double pref, double* A6, c128* h3,
                        cudaStream_t st);
void launch_q0avg_moments(int N, int nw, const c128* Y, c128* G, const double* A6, const double* dirs, int nd,
                          double* m, int* status, cudaStream_t st);
void launch_q0avg_update(int N, int nw, c128* X, long long sX, const c128* x1, const c128* G, const double* m,
                         cudaStream_t st);
// pair tables: delta[r] and (p.qhat)_{ia}(k) for r = ((kk*na)+a)*nb+b
void launch_pairs(int NK, int NBd, const int* nk, int q, int kk0, int nkk, int a0, int na, int b0, int nb,
                  const double* eps, const c128* pmom, const double* qhat, double* delta, float* delta_f,
                  c128* pq, cudaStream_t st);
// eps~(0) += (head - 1) x1 x1^H + x1 r + r^H x1^H, r = -c conj(Vb h)
void launch_q0_correction(int N, int nw, c128* eps_t, const c128* x1, const c128* Vbh, const double* head,
                          double c, cudaStream_t st);
void launch_midgap(int NK, int NBd, int nocc, const double* eps, double* mu, cudaStream_t st);

// k_sigma.cu
// S[r][j] = Re sum_nu U[r][nu] conj(a[r][nu])
template <typename T>
void launch_rowdot(int R, int N, const cplx<T>* U, const cplx<T>* a, long long ld, float* S_f, double* S_d, int j,
                   int nw, cudaStream_t st);
// sigma[k][n][w] += pref * sum_m sum_j g_j S[(kk,n,m)][j] 2z/(z^2+w_j^2), z = i w + mu - eps_m(k-q),
// for the target k = kk0 + kk of one chunk of rows r = ((kk*nsig)+n)*NBd + m.
void launch_sigma_conv_chunk(int kk0, int nkk, int nsig, int NBd, const int* nk, int q, const double* eps,
                             const double* mu, const float* S_f, const double* S_d, const double* freq,
                             const double* gw, int nw, double pref, c128* sigma, bool fp64, cudaStream_t st,
                             const int* ktab = nullptr);
// sigma[k] += part[k] for the target k the pass computed, part[-k] for the others (time reversal:
// Sigma_c(-k) = Sigma_c(k) when q -> 0 carries no direction); is_rep [NK]: 1 for computed k
void launch_sigma_trs_fill(int NK, int nsig, int nw, const int* nk, const int* is_rep, const c128* part,
                           c128* sigma, cudaStream_t st);
void launch_qp(int NK, int nsig, int NBd, int sig_lo, int nw, const c128* sigma, const double* dxv,
               const double* eps, const double* mu, const double* freq, double* e_qp, int* conv,
               cudaStream_t st);

// k_tc.cu -- tcgen05 split-precision Sigma_c contraction (and the chi0 / W^c plane helpers)
struct PlaneSet {
  void* b[6];       // B1 pieces then B2 pieces
};
struct TcSigmaArgs {
  int R;            // rows a_r = C^mu_{nm}(k, k-q) of this chunk
  int N;            // n_aux
  int Kpad;         // n_aux rounded up to 32 (K = mu)
  int nw;
  const float* raw; // [R][2*Kpad] fp32 (re, im) of a_r (zero beyond n_aux)
  const void* bpl[6];  // W^c planes [nw*N][2*Kpad] (B1 pieces then B2 pieces)
  void* apl[2];     // workspace: A pieces [R][2*Kpad] (bf16 or tf32), written by tc_sigma_run from raw
  float* S;         // [R][nw] accumulated (zeroed by the caller)
  int tf32;
  int* status;
};
gw_status tc_sigma_run(const TcSigmaArgs& a, cudaStream_t st, std::string& err);
// conj != 0: the planes of conj(W^c) (time reversal: W^c(-q) = conj(W^c(q)))
void tc_w_planes(int N, int nw, int Kpad, const c128* Wc, const PlaneSet& P, int tf32, cudaStream_t st, int conj = 0);
bool tc_available();
void tc_herm_fill(int N, int nw, c128* chi0, cudaStream_t st);

// k_chi0.cu -- tcgen05 chi0 with Re / Im rows stacked on the M side (all split precisions)
struct Chi0hArgs {
  int kind;                 // 0: FP16 two pieces (scaled), 1: BF16 three pieces, 2: TF32 two pieces
  int N, Kpad, T;           // n_aux, padded pair rows (multiple of 32), weight rows
  const float* raw;         // [N][2*Kpad] fp32 (re, im) of M
  void* bpl[3];             // B pieces [N][2*Kpad] (written by chi0h_pieces)
  const unsigned* absmax;   // largest |re|, |im| of raw (float bits)
  int* eB;                  // FP16: exponent of the B plane scale (device)
  float* wtab;              // [T][Kpad] weight rows (FP16: multiplied in place by their scales)
  double* escale;           // [T] device: factor of the drained sums
  double scale;             // -(s / N_k)
  c128* out;                // [T][N][N], lower triangle accumulated (caller zeroes it)
  int* status;
  int seg_rows;             // pair rows per FP64 promotion segment
  cudaEvent_t* events;      // NULL or two events recorded around the contraction launch
};
struct Chi0Plan;
void chi0_plan_free(Chi0Plan* p);
gw_status chi0h_pieces(const Chi0hArgs& a, cudaStream_t st);
gw_status chi0h_run(const Chi0hArgs& a, Chi0Plan** plan, cudaStream_t st, std::string& err);
// C[b] = alpha A[b] H[b] (b < nb; complex N x N row-major, N even; H[b] Hermitian) on the same
// tcgen05 kernel with unit weights, every element, TF32 two-piece operands, FP64 output (overwritten)
struct HermGemmArgs {
  int N, nb;
  const c64* A;          // [a_batch ? nb : 1][N][N]
  int a_batch;
  const c128* H64;       // [h_batch ? nb : 1][N][N] FP64, or NULL and H32 given
  const c64* H32;
  int h_batch;
  double alpha;
  c128* C;               // [nb][N][N]
  float* bpl[2];         // workspace: [(h_batch ? nb : 1) N][2 Kpad] fp32 each, Kpad = N rounded up to 32
  float* ones;           // workspace [Kpad]
  double* escale;        // workspace [nb]
  int* status;
};
gw_status herm_gemm_run(const HermGemmArgs& a, Chi0Plan** plan, cudaStream_t st, std::string& err);
// wtab[j][r] = 2 D_r / (w_j^2 + D_r^2) (0 for padding rows r >= K)
void chi0h_weights(int K, int Kpad, int nw, const float* delta, const double* freq, float* wtab, cudaStream_t st);

// Ritz modes and the surrogate reconstruction (k_modes.cu); small sizes nb <= 64
void launch_small_chol_linv(int nb, int batch, const c128* G, c128* Linv, int* status, cudaStream_t st);
void launch_small_jacobi(int nb, int batch, const c128* H, double* theta, c128* Z, cudaStream_t st);
void launch_mode_diag(int N, int k, int nc, const c128* U, const c128* T, long long sT, float* d, int ldd, int c0,
                      cudaStream_t st);
void launch_sur_inputs(int rows, int nc, const float* d, float* x, float* sig, cudaStream_t st);
void launch_sur_features(int rows, int nw, int j0, const int* jmap, const float* d, int nc, int nf, float* x,
                         float* y, cudaStream_t st);
void launch_freq_moments(int nw, long long NN, const c128* X, const int* cidx, const int* fidx, int nc, int nf,
                         double* gram, cudaStream_t st);
void launch_sur_coef(int rows, int nf, const float* sig, const float* g, float* coef, cudaStream_t st);
template <typename T>
void launch_sur_assemble(int R, int nc, int nw, int k, const int* jmap, const T* Sc, const cplx<T>* P,
                         const float* coef, int nf, const float* L, T* S, cudaStream_t st);

// frequency compression of chi0 (k_compress.cu)
void launch_wgram(int K, int nw, const double* delta, const double* freq, c128* G, cudaStream_t st);
void launch_wnorm(int nw, int batch, c128* G, double* nrm, cudaStream_t st);
void launch_wproj(int nw, int batch, const c128* Uh, const double* nrm, double* E, double* Pm, cudaStream_t st);
void launch_wresid(int K, int nw, const double* delta, const double* freq, const double* E, const double* Pm,
                   double* err, cudaStream_t st);
void launch_wtab_compressed(int K, int Kpad, int nw, int T, const double* delta, const double* freq, const double* Pm,
                            float* wtab, cudaStream_t st);
void launch_expand(int nw, int T, long long NN, const double* E, const c128* C, c128* chi0, cudaStream_t st);

// text returned by gw_last_error() on this thread
void gw_set_last_error(const std::string& msg);

// learned frequency surrogate (k_mlp.cu): g = s * MLP(x) for n <= 4096 rows on stream st
gw_status sur_correction(gw_surrogate_s* m, const float* x, int n, float* g_out, cudaStream_t st);
int sur_n_in(const gw_surrogate_s* m);
int sur_n_out(const gw_surrogate_s* m);
const float* sur_linear(const gw_surrogate_s* m);   // device [n_out][n_in] fp32

}  // namespace gw
