// Step (d): Sigma_c contraction and frequency convolution (Eq. GW_selfe_element with W^c),
// and the QP step: two-pole continuation + Newton solve of the quasiparticle equation.
#include "gw_internal.h"

namespace gw {

// S[r][j] = Re sum_nu U[r][nu] conj(a[r][nu]) -- one warp per row.
template <typename T>
__global__ void k_rowdot(int R, int N, const cplx<T>* __restrict__ U, const cplx<T>* __restrict__ a, long long ld,
                         float* S_f, double* S_d, int j, int nw) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
  if (warp >= R) return;
  const cplx<T>* u = U + (long long)warp * ld;
  const cplx<T>* v = a + (long long)warp * ld;
  double s = 0;
  for (int nu = lane; nu < N; nu += 32) s += (double)u[nu].re * v[nu].re + (double)u[nu].im * v[nu].im;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    if (S_d) S_d[(long long)warp * nw + j] = s;
    if (S_f) S_f[(long long)warp * nw + j] = (float)s;
  }
}
template <typename T>
void launch_rowdot(int R, int N, const cplx<T>* U, const cplx<T>* a, long long ld, float* S_f, double* S_d, int j,
                   int nw, cudaStream_t st) {
  int blocks = (R * 32 + 255) / 256;
  ++::gw::g_launch_count, k_rowdot<T><<<blocks, 256, 0, st>>>(R, N, U, a, ld, S_f, S_d, j, nw);
}
template void launch_rowdot<double>(int, int, const c128*, const c128*, long long, float*, double*, int, int,
                                    cudaStream_t);
template void launch_rowdot<float>(int, int, const c64*, const c64*, long long, float*, double*, int, int,
                                   cudaStream_t);

// sigma[k][n][w] += pref * sum_m sum_j g_j S[(kk,n,m)][j] 2 z / (z^2 + w_j^2),  z = i w + mu - eps_m(k - q)
// Rows of S are r = ((kk * nsig) + n) * NBd + m for k = kk0 + kk. One thread per (kk, n, w).
template <typename T>
__global__ void k_sigma_conv(int nkk, int kk0, int nsig, int NBd, int n1, int n2, int n3, int q,
                             const double* __restrict__ eps, const double* __restrict__ mu_p,
                             const float* __restrict__ S_f, const double* __restrict__ S_d,
                             const double* __restrict__ freq, const double* __restrict__ gw, int nw, double pref,
                             c128* __restrict__ sigma, const int* __restrict__ ktab) {
  extern __shared__ double sh[];
  double* fr = sh;
  double* gg = sh + nw;
  for (int i = threadIdx.x; i < nw; i += blockDim.x) {
    fr[i] = freq[i];
    gg[i] = gw[i];
  }
  __syncthreads();
  const int total = nkk * nsig * nw;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int w_i = t % nw, n = (t / nw) % nsig, kk = t / (nw * nsig);
  const int k = ktab ? ktab[kk0 + kk] : kk0 + kk;
  int k3 = k % n3, k2 = (k / n3) % n2, k1 = k / (n2 * n3);
  int q3 = q % n3, q2 = (q / n3) % n2, q1 = q / (n2 * n3);
  int kmq = (((k1 - q1 + n1) % n1) * n2 + ((k2 - q2 + n2) % n2)) * n3 + ((k3 - q3 + n3) % n3);
  const T om = (T)fr[w_i];
  const T mu = (T)*mu_p;
  T acc_re = 0, acc_im = 0;
  for (int m = 0; m < NBd; ++m) {
    const long long r = ((long long)kk * nsig + n) * NBd + m;
    const T zr = mu - (T)eps[(long long)kmq * NBd + m];   // z = zr + i om
    // z^2 = zr^2 - om^2 + 2 i zr om
    const T z2r = zr * zr - om * om, z2i = (T)2 * zr * om;
    T sr = 0, si = 0;
    for (int j = 0; j < nw; ++j) {
      const T s = (T)gg[j] * (S_d ? (T)S_d[r * nw + j] : (T)S_f[r * nw + j]);
      const T wj = (T)fr[j];
      // 2 z / (z^2 + wj^2)
      const T dr = z2r + wj * wj, di = z2i;
      const T inv = (T)1 / (dr * dr + di * di);
      const T fr_ = (T)2 * (zr * dr + om * di) * inv;
      const T fi_ = (T)2 * (om * dr - zr * di) * inv;
      sr += s * fr_;
      si += s * fi_;
    }
    acc_re += sr;
    acc_im += si;
  }
  c128* o = sigma + ((long long)k * nsig + n) * nw + w_i;
  o->re += pref * (double)acc_re;
  o->im += pref * (double)acc_im;
}

void launch_sigma_conv_chunk(int kk0, int nkk, int nsig, int NBd, const int* nk, int q, const double* eps,
                             const double* mu, const float* S_f, const double* S_d, const double* freq,
                             const double* gw, int nw, double pref, c128* sigma, bool fp64, cudaStream_t st,
                             const int* ktab) {
  int total = nkk * nsig * nw;
  size_t smem = 2 * nw * sizeof(double);
  if (fp64)
    ++::gw::g_launch_count, k_sigma_conv<double><<<(total + 127) / 128, 128, smem, st>>>(nkk, kk0, nsig, NBd, nk[0], nk[1], nk[2], q, eps,
                                                                 mu, S_f, S_d, freq, gw, nw, pref, sigma, ktab);
  else
    ++::gw::g_launch_count, k_sigma_conv<float><<<(total + 127) / 128, 128, smem, st>>>(nkk, kk0, nsig, NBd, nk[0], nk[1], nk[2], q, eps,
                                                                mu, S_f, S_d, freq, gw, nw, pref, sigma, ktab);
}

__global__ void k_sigma_trs_fill(int NK, int nsig, int nw, int n1, int n2, int n3, const int* __restrict__ is_rep,
                                 const c128* __restrict__ part, c128* __restrict__ sigma) {
  const long long per_k = (long long)nsig * nw;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)NK * per_k;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e / per_k);
    int src = k;
    if (!is_rep[k]) {
      const int k3 = k % n3, k2 = (k / n3) % n2, k1 = k / (n2 * n3);
      src = (((n1 - k1) % n1) * n2 + (n2 - k2) % n2) * n3 + (n3 - k3) % n3;
    }
    const c128 v = part[(long long)src * per_k + e % per_k];
    sigma[e].re += v.re;
    sigma[e].im += v.im;
  }
}
void launch_sigma_trs_fill(int NK, int nsig, int nw, const int* nk, const int* is_rep, const c128* part,
                           c128* sigma, cudaStream_t st) {
  const long long total = (long long)NK * nsig * nw;
  ++::gw::g_launch_count, k_sigma_trs_fill<<<(int)std::min<long long>((total + 255) / 256, 152LL * 8), 256, 0, st>>>(
      NK, nsig, nw, nk[0], nk[1], nk[2], is_rep, part, sigma);
}

// ---------------------------------------------------------------------------------------------
// QP: two-pole model Sigma(z) = (p1 z + p0) / (z^2 + q1 z + q0) from the linear least-squares
// problem f_j z_j^2 = -q1 f_j z_j - q0 f_j + p1 z_j + p0 over all frequencies (columns scaled
// to unit norm, solved by modified Gram-Schmidt QR applied twice), then Newton on
// E = eps_n + Re Sigma(E - mu) + dxv. One thread per (k, n).
// ---------------------------------------------------------------------------------------------
constexpr int QP_MAXW = 256;

__device__ __forceinline__ c128 cdiv(c128 a, c128 b) {
  double d = b.re * b.re + b.im * b.im;
  return c128{(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

__global__ void k_qp(int NK, int nsig, int NBd, int sig_lo, int nw, const c128* __restrict__ sigma,
                     const double* __restrict__ dxv, const double* __restrict__ eps, const double* __restrict__ mu_p,
                     const double* __restrict__ freq, double* e_qp, int* conv) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NK * nsig) return;
  const int k = t / nsig, n = t % nsig;
  const c128* f = sigma + (long long)t * nw;
  // columns of A: [-f z, -f, z, 1], rhs b = f z^2 (z = i w_j)
  c128 Q[4][QP_MAXW];
  c128 b[QP_MAXW];
  double scale[4];
  for (int j = 0; j < nw; ++j) {
    const c128 z = c128{0.0, freq[j]};
    const c128 fj = f[j];
    const c128 fz = cmul(fj, z);
    Q[0][j] = c128{-fz.re, -fz.im};
    Q[1][j] = c128{-fj.re, -fj.im};
    Q[2][j] = z;
    Q[3][j] = c128{1.0, 0.0};
    b[j] = cmul(fz, z);
  }
  for (int c = 0; c < 4; ++c) {
    double s = 0;
    for (int j = 0; j < nw; ++j) s += Q[c][j].re * Q[c][j].re + Q[c][j].im * Q[c][j].im;
    scale[c] = sqrt(s);
    for (int j = 0; j < nw; ++j) Q[c][j] = c128{Q[c][j].re / scale[c], Q[c][j].im / scale[c]};
  }
  c128 Rm[4][4];
  for (int i = 0; i < 4; ++i)
    for (int c = 0; c < 4; ++c) Rm[i][c] = c128{0, 0};
  for (int c = 0; c < 4; ++c) {
    for (int pass = 0; pass < 2; ++pass) {
      for (int i = 0; i < c; ++i) {
        c128 d = {0, 0};  // Q_i^H Q_c
        for (int j = 0; j < nw; ++j) d = cadd(d, cmulc(Q[c][j], Q[i][j]));
        Rm[i][c] = cadd(Rm[i][c], d);
        for (int j = 0; j < nw; ++j) {
          c128 p = cmul(d, Q[i][j]);
          Q[c][j] = c128{Q[c][j].re - p.re, Q[c][j].im - p.im};
        }
      }
    }
    double s = 0;
    for (int j = 0; j < nw; ++j) s += Q[c][j].re * Q[c][j].re + Q[c][j].im * Q[c][j].im;
    s = sqrt(s);
    Rm[c][c] = c128{s, 0};
    for (int j = 0; j < nw; ++j) Q[c][j] = c128{Q[c][j].re / s, Q[c][j].im / s};
  }
  c128 y[4];
  for (int i = 0; i < 4; ++i) {
    c128 d = {0, 0};
    for (int j = 0; j < nw; ++j) d = cadd(d, cmulc(b[j], Q[i][j]));
    y[i] = d;
  }
  c128 x[4];
  for (int i = 3; i >= 0; --i) {
    c128 s = y[i];
    for (int c = i + 1; c < 4; ++c) {
      c128 p = cmul(Rm[i][c], x[c]);
      s = c128{s.re - p.re, s.im - p.im};
    }
    x[i] = cdiv(s, Rm[i][i]);
  }
  const c128 q1 = c128{x[0].re / scale[0], x[0].im / scale[0]};
  const c128 q0 = c128{x[1].re / scale[1], x[1].im / scale[1]};
  const c128 p1 = c128{x[2].re / scale[2], x[2].im / scale[2]};
  const c128 p0 = c128{x[3].re / scale[3], x[3].im / scale[3]};
  const double mu = *mu_p;
  const double e0 = eps[(long long)k * NBd + sig_lo + n];
  const double dx = dxv ? dxv[t] : 0.0;
  auto val_der = [&](double xr, double& v, double& d) {
    const c128 X = c128{xr, 0.0};
    const c128 num = cadd(cmul(p1, X), p0);
    const c128 den = cadd(cadd(cmul(X, X), cmul(q1, X)), q0);
    const c128 dnum = p1;
    const c128 dden = cadd(c128{2.0 * xr, 0.0}, q1);
    v = cdiv(num, den).re;
    const c128 top = c128{cmul(dnum, den).re - cmul(num, dden).re, cmul(dnum, den).im - cmul(num, dden).im};
    d = cdiv(top, cmul(den, den)).re;
  };
  double E = e0;
  int ok = 0;
  for (int it = 0; it < 100; ++it) {
    double v, d;
    val_der(E - mu, v, d);
    const double step = (E - e0 - v - dx) / (1.0 - d);
    E -= step;
    if (!isfinite(E)) break;
    if (fabs(step) < 1e-10) {
      ok = 1;
      break;
    }
  }
  if (!ok) {
    double v, d;
    val_der(e0 - mu, v, d);
    E = e0 + (v + dx) / (1.0 - d);
  }
  e_qp[t] = E;
  conv[t] = ok;
}

void launch_qp(int NK, int nsig, int NBd, int sig_lo, int nw, const c128* sigma, const double* dxv, const double* eps,
               const double* mu, const double* freq, double* e_qp, int* conv, cudaStream_t st) {
  int total = NK * nsig;
  ++::gw::g_launch_count, k_qp<<<(total + 63) / 64, 64, 0, st>>>(NK, nsig, NBd, sig_lo, nw, sigma, dxv, eps, mu, freq, e_qp, conv);
}

}  // namespace gw
