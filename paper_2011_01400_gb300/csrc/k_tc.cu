// Tensor-core (tcgen05) split-precision contraction of step (d), Eq. GW_selfe_element with W^c:
//   U_{r nu} = sum_mu a_{r mu} W^c_{mu nu}(w') = sum_mu a_{r mu} conj(W^c_{nu mu})  (W^c Hermitian),
//   S_r(w') = Re sum_nu U_{r nu} conj(a_{r nu}),  a_r = C^mu_{nm}(k, k-q);
// the row dot is fused into the epilogue and accumulated into S[r][w'].
//
// Every operand row interleaves (re, im) along K. Real form of one complex product:
//   Re U = A . B1^T,  B1 = (w_re, w_im);   Im U = A . B2^T,  B2 = (-w_im, w_re),
// so one MMA against the stacked operand [B1; B2] (N = 2 x 64) yields Re and Im columns.
// Operands are split into two pieces (BF16 or TF32: h + l); hh, hl and lh are accumulated. The A
// pieces are split before the launch (k_a_planes) and streamed by TMA like the B pieces.
//
// Accumulation. The tensor-core FP32 accumulator rounds every addition toward zero. hh goes to
// accumulator D1, the correction products (2^-8 smaller) to D2; both are drained once per segment
// into FP32 running sums held in registers by the epilogue warps (K = n_aux is short: at most 52
// MMAs per item, a truncation bias ~1e-6 relative of S, far inside the Sigma_c tolerance).
//
// Hermitian triangle: column block nb needs K = mu from its own block on; the block's own 64
// ABFs form one segment (counted once), the rest a second one (counted twice, 2 Re).
//
// Work distribution: one CTA per SM, each walking the work items (row block, frequency, column
// block; column block fastest, so that concurrent CTAs share their W^c tiles in L2); all
// pipelines (barrier phases, TMEM buffers) run on across items.
//
// Roles (384 threads):
//   * warp 0 (TMA):   B1 / B2 pieces, 64 rows x 128 B each per stage, SWIZZLE_128B
//   * warp 2 (TMA):   A pieces, 128 rows x 128 B each per stage; after each item's stages the
//                     item's fp32 a tile (128 rows x BN complex) into the a-tile buffer for the
//                     epilogue's row dot
//   * warp 1:         one elected thread issues tcgen05.mma (M = 128, N = 128) into TMEM
//   * warps 4-11:     epilogue (two warps per TMEM lane quadrant, 32 complex columns each)
// All mbarrier waits are bounded; on expiry the kernel sets ST_TIMEOUT and unwinds.
#include "gw_internal.h"
#include "tc_ptx.cuh"

#include <cuda.h>
#include <cuda_bf16.h>

#include <cstdlib>
#include <vector>

namespace gw {

namespace {

using namespace ptx;

constexpr int BM = 128, BN = 64;                   // complex output tile
constexpr int TILE = 128 * ROWB;                   // 16 KB: A piece (128 rows) or B piece ([B1; B2], 128 rows)
constexpr int HALF = 64 * ROWB;                    // 8 KB: B1 or B2 part of a B piece
constexpr int RAW = 128 * ROWB;                    // 16 KB: one fp32 box (32 floats x 128 rows) of the a tile
constexpr int RAW_BOXES = 2 * BN / 32;             // boxes of one BN-column a tile
constexpr int NP = 2;                              // pieces per operand
constexpr int NTHREADS = 384;
// TMEM columns: D1 buffers at 0 and 128 (re: +0..63, im: +64..127); D2 buffers at 256 and 384
constexpr uint32_t D1_COL = 0, D2_COL = 256, DBUF = 128;

template <bool TF32> struct Cfg {
  static constexpr int STAGE = 2 * NP * TILE;      // B pieces then A pieces
  static constexpr int STAGES = 2;
  static constexpr int RS = TF32 ? 16 : 32;        // complex K entries per stage (128 B rows)
  static constexpr int BAR_OFF = STAGES * STAGE + RAW_BOXES * RAW;
  static constexpr int SMEM = BAR_OFF + 256 + 1024;
};
static_assert(Cfg<false>::SMEM <= 232448 && Cfg<true>::SMEM <= 232448, "shared memory budget");

// sr[j] += D[re column t + j], si[j] += D[im column t + BN + j], j < 32, sixteen columns at a time
// (keeps the running sums and one half of the drained columns in registers)
__device__ __forceinline__ void drain_add(uint32_t t, float (&sr)[32], float (&si)[32]) {
  uint32_t vr[16], vi[16], wr[16], wi[16];
  tmem_ld16_nowait(t, vr);
  tmem_ld16_nowait(t + BN, vi);
  tmem_ld16_nowait(t + 16, wr);
  tmem_ld16_nowait(t + BN + 16, wi);
  tmem_wait_ld();
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    sr[j] += __uint_as_float(vr[j]);
    si[j] += __uint_as_float(vi[j]);
    sr[16 + j] += __uint_as_float(wr[j]);
    si[16 + j] += __uint_as_float(wi[j]);
  }
}


struct TcParams {
  int Mrows, Ncols;   // A rows r, B rows nu
  int nstage;         // stages over K = mu
  int n_items, nw, nnb;
  float* S;           // [Mrows][nw]
  int* status;
};

struct Maps {
  CUtensorMap b[4];   // B1 pieces then B2 pieces
  CUtensorMap raw;    // A-side fp32 plane, 32 floats x 128 rows per box (the row dot's a tile)
  CUtensorMap a[2];   // A-side pieces (128 B x 128 rows per box)
};

__device__ __forceinline__ void decode_item(const TcParams& p, int item, int& m0, int& n0, int& w) {
  const int nb = item % p.nnb;
  const int rest = item / p.nnb;
  w = rest % p.nw;
  m0 = (rest / p.nw) * BM;
  n0 = nb * BN;
}

// the triangle's K range of column block n0 and its two segments
template <int RS>
__device__ __forceinline__ int first_stage(int n0) { return n0 / RS; }
template <int RS>
__device__ __forceinline__ bool is_seg_first(int i, int i0) { return i == i0 || i == i0 + BN / RS; }
template <int RS>
__device__ __forceinline__ bool is_seg_end(int i, int i0, int nst) { return i == nst - 1 || i == i0 + BN / RS - 1; }

template <bool TF32>
__global__ void __launch_bounds__(NTHREADS, 1) k_tc(const __grid_constant__ Maps maps, TcParams p) {
  using C = Cfg<TF32>;
  constexpr int STAGES = C::STAGES, STAGE = C::STAGE, RS = C::RS;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* atile = smem + STAGES * STAGE;    // the item's fp32 a tile: RAW_BOXES boxes
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::BAR_OFF);
  uint64_t* full_b = bars;                   // [STAGES]
  uint64_t* full_a = bars + STAGES;          // [STAGES]
  uint64_t* empty = bars + 2 * STAGES;       // [STAGES]
  uint64_t* t1full = bars + 3 * STAGES;      // [2] D1 of a segment ready
  uint64_t* t1empty = bars + 3 * STAGES + 2; // [2] D1 drained
  uint64_t* t2full = bars + 3 * STAGES + 4;  // [2] D2 of a segment ready
  uint64_t* t2empty = bars + 3 * STAGES + 6; // [2] D2 drained
  uint64_t* done = bars + 3 * STAGES + 8;
  uint64_t* tfull = bars + 3 * STAGES + 9;   // the a tile landed
  uint64_t* tempty = bars + 3 * STAGES + 10; // the a tile read by the epilogue
  uint32_t* tmem_base_p = reinterpret_cast<uint32_t*>(bars + 3 * STAGES + 11);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_b[s], 1);
      mbar_init(&full_a[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&t1full[b], 1);
      mbar_init(&t1empty[b], 8);                // one per epilogue warp
      mbar_init(&t2full[b], 1);
      mbar_init(&t2empty[b], 8);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, 8);
    mbar_init(done, 1);
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_base_p, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_base_p;
  const int nst = p.nstage;

  if (warp == 0) {
    // ---------------- TMA producer: B1 / B2 pieces ----------------
    if (lane == 0) {
      uint32_t gs = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
        int m0, n0, w;
        decode_item(p, item, m0, n0, w);
        const int yrow = w * p.Ncols + n0;
        for (int i = first_stage<RS>(n0); i < nst; ++i, ++gs) {
          const int s = gs % STAGES;
          if (!mbar_wait(&empty[s], ((gs / STAGES) & 1) ^ 1, p.status)) { ok = false; break; }
          uint8_t* st = smem + s * STAGE;
          mbar_arrive_expect_tx(&full_b[s], NP * TILE);
          const int x = i * (ROWB / (TF32 ? 4 : 2));
#pragma unroll
          for (int pc = 0; pc < NP; ++pc) {
            tma_load_2d(st + pc * TILE, &maps.b[pc], &full_b[s], x, yrow);              // B1 rows 0..63
            tma_load_2d(st + pc * TILE + HALF, &maps.b[NP + pc], &full_b[s], x, yrow);  // B2 rows 64..127
          }
        }
      }
    }
  } else if (warp == 2) {
    // ---------------- TMA producer: A pieces into the stages, then the item's a tile ----------------
    if (lane == 0) {
      uint32_t gs = 0, gt = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
        int m0, n0, w;
        decode_item(p, item, m0, n0, w);
        for (int i = first_stage<RS>(n0); i < nst; ++i, ++gs) {
          const int s = gs % STAGES;
          if (!mbar_wait(&empty[s], ((gs / STAGES) & 1) ^ 1, p.status)) { ok = false; break; }
          uint8_t* at = smem + s * STAGE + NP * TILE;
          mbar_arrive_expect_tx(&full_a[s], NP * TILE);
          const int x = i * (ROWB / (TF32 ? 4 : 2));
#pragma unroll
          for (int pc = 0; pc < NP; ++pc) tma_load_2d(at + pc * TILE, &maps.a[pc], &full_a[s], x, m0);
        }
        if (ok) {
          // the fp32 a tile of the epilogue's row dot (rows m0.., columns n0..n0+BN-1): issued after
          // the item's stages, since it is read only at the item's end, once the previous item's
          // epilogue has released the buffer
          if (!mbar_wait(tempty, (gt & 1) ^ 1, p.status)) break;
          mbar_arrive_expect_tx(tfull, RAW_BOXES * RAW);
#pragma unroll
          for (int c = 0; c < RAW_BOXES; ++c) tma_load_2d(atile + c * RAW, &maps.raw, tfull, 2 * n0 + 32 * c, m0);
          ++gt;
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      constexpr uint32_t fmt = TF32 ? 2u : 1u;
      const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)((2 * BN) >> 3) << 17) |
                             ((uint32_t)(BM >> 4) << 24);
      uint32_t gs = 0, gseg = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
        int m0, n0, w;
        decode_item(p, item, m0, n0, w);
        const int i0 = first_stage<RS>(n0);
        for (int i = i0; i < nst; ++i, ++gs) {
          const int s = gs % STAGES;
          const int b = gseg & 1;
          const bool seg_first = is_seg_first<RS>(i, i0);
          if (seg_first && gseg >= 2 && !mbar_wait(&t1empty[b], ((gseg >> 1) - 1) & 1, p.status)) {
            ok = false;
            break;
          }
          if (seg_first && gseg >= 2 && !mbar_wait(&t2empty[b], ((gseg >> 1) - 1) & 1, p.status)) {
            ok = false;
            break;
          }
          if (!mbar_wait(&full_b[s], (gs / STAGES) & 1, p.status)) { ok = false; break; }
          if (!mbar_wait(&full_a[s], (gs / STAGES) & 1, p.status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t bbase = smem_u32(smem + s * STAGE);
          const uint32_t abase = bbase + NP * TILE;
          const uint32_t d1 = tmem + D1_COL + b * DBUF;
          const uint32_t d2 = tmem + D2_COL + b * DBUF;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint32_t ko = kk * 32;
            const uint32_t acc = (seg_first && kk == 0) ? 0u : 1u;
            const uint64_t A0 = sdesc(abase + ko), B0 = sdesc(bbase + ko);
            const uint64_t A1 = sdesc(abase + TILE + ko), B1 = sdesc(bbase + TILE + ko);
            mma<TF32>(d1, A0, B0, idesc, acc);
            mma<TF32>(d2, A0, B1, idesc, acc);
            mma<TF32>(d2, A1, B0, idesc, 1u);
          }
          mma_commit(&empty[s]);
          if (is_seg_end<RS>(i, i0, nst)) {
            mma_commit(&t1full[b]);
            mma_commit(&t2full[b]);
            ++gseg;
          }
        }
      }
      mma_commit(done);
      mbar_wait(done, 0, p.status);
    }
  } else if (warp >= 4 && warp <= 11) {
    // ---------------- epilogue: drain D1 and D2 per segment, row dot ----------------
    const int quad = warp & 3;                 // TMEM lanes 32*quad .. 32*quad+31
    const int half = (warp - 4) >> 2;          // output columns half*32 .. half*32+31
    const int row = quad * 32 + lane;
    const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
    uint32_t gseg = 0, gt = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
      int m0, n0, w;
      decode_item(p, item, m0, n0, w);
      const int m = m0 + row;
      const int c0 = n0 + half * 32;
      const int i0 = first_stage<RS>(n0);
      bool tile_ready = false;
      float sr[32], si[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) sr[j] = si[j] = 0.f;
      for (int i = i0; i < nst; ++i) {
        if (!is_seg_end<RS>(i, i0, nst)) continue;
        const int b = gseg & 1;
        const uint32_t ph = (gseg >> 1) & 1;
        // every lane polls the barrier; reconverge before the warp-wide (.sync.aligned) TMEM loads
        ok = __all_sync(0xffffffffu, mbar_wait(&t1full[b], ph, p.status));
        if (!ok) break;
        tc_fence_after();
        drain_add(tmem + lane_off + D1_COL + b * DBUF + half * 32, sr, si);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&t1empty[b]);
        ok = __all_sync(0xffffffffu, mbar_wait(&t2full[b], ph, p.status));
        if (!ok) break;
        tc_fence_after();
        drain_add(tmem + lane_off + D2_COL + b * DBUF + half * 32, sr, si);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&t2empty[b]);
        ++gseg;
        const int nmax = p.Ncols - c0;
        if (!tile_ready) {
          ok = __all_sync(0xffffffffu, mbar_wait(tfull, gt & 1, p.status));
          if (!ok) break;
          tile_ready = true;
        }
        if (m < p.Mrows) {
          // S_r += Re sum_nu U_{r nu} conj(a_{r nu}) over this thread's 32 columns, a from the a
          // tile (complex column 32 half + j: box 2 half + j / 16, 16-B chunk (j % 16) / 2)
          float acc = 0.f;
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const float4 a = *reinterpret_cast<const float4*>(atile + (2 * half + jj / 8) * RAW + swz(row, jj % 8));
            if (2 * jj < nmax) acc = fmaf(sr[2 * jj], a.x, fmaf(si[2 * jj], a.y, acc));
            if (2 * jj + 1 < nmax) acc = fmaf(sr[2 * jj + 1], a.z, fmaf(si[2 * jj + 1], a.w, acc));
          }
          // the diagonal block counts once, the strictly lower blocks twice (2 Re)
          const float wgt = (i > i0 + (BN / RS) - 1) ? 2.f : 1.f;
          atomicAdd(p.S + (long long)m * p.nw + w, wgt * acc);
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) sr[j] = si[j] = 0.f;
        if (i == nst - 1) {
          // last segment of the item: release the a tile (generic reads before the TMA refill)
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) mbar_arrive(tempty);
          ++gt;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, 512);
}

// chi0[w][i][j] = conj(chi0[w][j][i]) for i < j (the kernel writes lower tiles only)
__global__ void k_herm_fill(int N, int nw, c128* chi0) {
  const long long total = (long long)nw * N * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % N), i = (int)((e / N) % N);
    const long long w = e / ((long long)N * N);
    if (i < j) {
      const c128 v = chi0[(w * N + j) * N + i];
      chi0[(w * N + i) * N + j] = c128{v.re, -v.im};
    }
  }
}

// A pieces of an fp32 (re, im) plane [rows][ldk] for the pre-split path, two pieces:
// BF16: h = bf16(y), l = bf16(y - h);  TF32: h = tf32(y), l = y - h (read as TF32 by the MMA).
__global__ void k_a_planes(long long n, const float* __restrict__ raw, void* p0, void* p1, int tf32) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float2 y = reinterpret_cast<const float2*>(raw)[e];
    if (tf32) {
      const float hr = tf32_rn(y.x), hi = tf32_rn(y.y);
      reinterpret_cast<float2*>(p0)[e] = make_float2(hr, hi);
      reinterpret_cast<float2*>(p1)[e] = make_float2(y.x - hr, y.y - hi);
    } else {
      const __nv_bfloat162 hh = __floats2bfloat162_rn(y.x, y.y);
      const float2 hf = __bfloat1622float2(hh);
      reinterpret_cast<__nv_bfloat162*>(p0)[e] = hh;
      reinterpret_cast<__nv_bfloat162*>(p1)[e] = __floats2bfloat162_rn(y.x - hf.x, y.y - hf.y);
    }
  }
}

// B planes of W^c (conj: of conj(W^c)) for the Sigma contraction: row (j, nu), K index 2 mu + {0, 1}:
// B1 = split(Re W_{nu mu}, Im W_{nu mu}), B2 = split(-Im, Re); mu >= N is zero padding.
__global__ void k_w_planes(int N, int nw, int Kpad, const c128* __restrict__ Wc, PlaneSet P, int tf32, int np,
                           int conj) {
  const long long total = (long long)nw * N * Kpad;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int mu = (int)(e % Kpad);
    const long long row = e / Kpad;                 // j * N + nu
    float v1[2] = {0.f, 0.f};
    if (mu < N) {
      const c128 w = Wc[row * N + mu];
      v1[0] = (float)w.re;
      v1[1] = conj ? -(float)w.im : (float)w.im;
    }
    const float v2[2] = {-v1[1], v1[0]};
    const long long o = row * 2LL * Kpad + 2LL * mu;
    for (int half = 0; half < 2; ++half) {
      const float* v = half ? v2 : v1;
      if (tf32) {
        const float h0 = tf32_rn(v[0]), h1 = tf32_rn(v[1]);
        *reinterpret_cast<float2*>(reinterpret_cast<float*>(P.b[2 * half]) + o) = make_float2(h0, h1);
        *reinterpret_cast<float2*>(reinterpret_cast<float*>(P.b[2 * half + 1]) + o) = make_float2(v[0] - h0, v[1] - h1);
      } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[0], v[1]);
        const float2 hf = __bfloat1622float2(h);
        const float r0 = v[0] - hf.x, r1 = v[1] - hf.y;
        const __nv_bfloat162 mm = __floats2bfloat162_rn(r0, r1);
        *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(P.b[np * half]) + o) = h;
        *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(P.b[np * half + 1]) + o) = mm;
        if (np == 3) {
          const float2 mf = __bfloat1622float2(mm);
          const __nv_bfloat162 l = __floats2bfloat162_rn(r0 - mf.x, r1 - mf.y);
          *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(P.b[np * half + 2]) + o) = l;
        }
      }
    }
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2-D map over a row-major plane [rows][ldk] of 16-bit (bf16) or 32-bit (fp32/tf32) elements,
// box = 128 B of one row x box_rows rows, 128-byte swizzle.
bool make_map(CUtensorMap* m, const void* base, int four_byte, long long ldk, long long rows, int box_rows,
              std::string& err) {
  EncodeTiledFn enc = get_encode();
  if (!enc) {
    err = "cuTensorMapEncodeTiled is unavailable";
    return false;
  }
  const int esz = four_byte ? 4 : 2;
  cuuint64_t dims[2] = {(cuuint64_t)ldk, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ldk * esz)};
  cuuint32_t box[2] = {(cuuint32_t)(ROWB / esz), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, four_byte ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                   const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
    return false;
  }
  return true;
}

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
  }
  return n;
}

template <bool TF32>
gw_status launch_tc(const Maps& maps, const TcParams& p, cudaStream_t st, std::string& err) {
  const int smem = Cfg<TF32>::SMEM;
  cudaFuncSetAttribute(k_tc<TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  const int grid = std::min(p.n_items, num_sms());
  ++::gw::g_launch_count, k_tc<TF32><<<grid, NTHREADS, smem, st>>>(maps, p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = std::string("k_tc launch: ") + cudaGetErrorString(e);
    return GW_ERR_CUDA;
  }
  return GW_OK;
}

}  // namespace

bool tc_available() { return get_encode() != nullptr; }

gw_status tc_sigma_run(const TcSigmaArgs& a, cudaStream_t st, std::string& err) {
  const bool tf32 = a.tf32 != 0;
  // Sigma_c needs ~1e-5 relative accuracy: two pieces per operand (hh, hl, lh) in both kinds
  const int RS = tf32 ? Cfg<true>::RS : Cfg<false>::RS;
  if (a.Kpad % 32 != 0) {
    err = "tc_sigma: Kpad must be a multiple of 32";
    return GW_ERR_ARG;
  }
  if (!a.apl[0] || !a.apl[1]) {
    err = "tc_sigma: the A piece workspace is NULL";
    return GW_ERR_ARG;
  }
  const int nmb = (a.R + BM - 1) / BM, nnb = (a.N + BN - 1) / BN;
  const long long items = (long long)nmb * nnb * a.nw;
  if (items > 0x7fffffffLL) {
    err = "tc_sigma: too many work items";
    return GW_ERR_ARG;
  }
  Maps maps;
  const long long ldk = 2LL * a.Kpad;
  for (int i = 0; i < 2 * NP; ++i)
    if (!make_map(&maps.b[i], a.bpl[i], tf32, ldk, (long long)a.nw * a.N, BN, err)) return GW_ERR_CUDA;
  if (!make_map(&maps.raw, a.raw, 1, ldk, a.R, BM, err)) return GW_ERR_CUDA;
  const long long n = (long long)a.R * a.Kpad;   // complex elements
  ++::gw::g_launch_count, k_a_planes<<<std::min<long long>((n + 255) / 256, 152 * 64), 256, 0, st>>>(
      n, a.raw, a.apl[0], a.apl[1], tf32 ? 1 : 0);
  for (int i = 0; i < NP; ++i)
    if (!make_map(&maps.a[i], a.apl[i], tf32, ldk, a.R, BM, err)) return GW_ERR_CUDA;
  TcParams p{};
  p.Mrows = a.R;
  p.Ncols = a.N;
  p.nstage = a.Kpad / RS;
  p.n_items = (int)items;
  p.nw = a.nw;
  p.nnb = nnb;
  p.S = a.S;
  p.status = a.status;
  return tf32 ? launch_tc<true>(maps, p, st, err) : launch_tc<false>(maps, p, st, err);
}

void tc_w_planes(int N, int nw, int Kpad, const c128* Wc, const PlaneSet& P, int tf32, cudaStream_t st, int conj) {
  const long long total = (long long)nw * N * Kpad;
  ++::gw::g_launch_count, k_w_planes<<<std::min<long long>((total + 255) / 256, 152 * 64), 256, 0, st>>>(N, nw, Kpad, Wc, P, tf32, 2, conj);
}

void tc_herm_fill(int N, int nw, c128* chi0, cudaStream_t st) {
  const long long total = (long long)nw * N * N;
  ++::gw::g_launch_count, k_herm_fill<<<std::min<long long>((total + 255) / 256, 152 * 64), 256, 0, st>>>(N, nw, chi0);
}

}  // namespace gw
