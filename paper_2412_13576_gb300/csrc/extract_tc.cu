// Algorithm 2 (§3.2) on the 5th-generation tensor cores: one persistent
// kernel runs all T Adam steps; each CTA owns 64 starts for the whole run.
//
// Per step, with B in shared memory as BF16 (exact: |B_ij| <= 256), and
// hi = bf16(z), lo = bf16(z - hi) (z carried to ~16 significant bits, so that
// B z is as accurate as an FP32 dot product; hi alone is the faster and
// coarser MAPE_PREC_BF16X1):
//   forward  B hi(z) + B lo(z), and g = B bf16(round z) of the previous step's
//            iterate (exact: |round z| <= 256 is exact in BF16, every partial
//            sum is an integer below 2^24 and FP32 accumulation is exact)
//   S = sign(B z) as BF16 {-1, 0, 1} in shared memory
//   G = S . B      (M = 64 starts, N = d_pad, K = n_pad rows of B), B read
//            through an MN-major descriptor of the forward tile (or a
//            transposed K-major copy when it fits)
//   grad = G + lambda1 (ceil z + floor z - 2 z) + the inverse-norm term; Adam
//   on the FP32 master z, m, v, held for the whole run in TMEM lanes 16-31
//   of each 32-lane quarter (the lanes an M = 64 accumulator leaves free: z,
//   m, v in columns [0, d), [d, 2d), [2d, 3d)) when 3 d_pad <= 512, else
//   blocked [tile][d/4][64][4] in global memory (L2 resident); the new
//   bf16(z) and bf16(round z) operands are written for the next step.
// The forward product takes one of two forms.  For tiles of at most 64 rows
// of B it is transposed: one MMA chain D^T = B_tile . [hi(Z); lo(Z); round(Z)]^T
// (M = 64 rows of B, N = 64 starts per operand tile, K = d_pad), so that TMEM
// lane i holds row i of B for every start and S is written MN-major; that is
// 10 MMA instructions for d = 160 instead of 30 (an MMA instruction costs
// about the same whatever its M and N).  Otherwise start r is row r of
// D1 = hi(Z) . B^T + lo(Z) . B^T and D2 = bf16(round Z) . B^T (M = 64,
// N = n_pad).  Row r of an M = 64 accumulator is TMEM lane 32 (r / 16) + r % 16
// (lanes 0-15 of each quarter).  The candidate of step t (D2 of step t + 1)
// is tested (C4, nonzero), signed canonically and appended while the
// gradient MMA runs.
//
// 16 warps: warp w reads TMEM lane quarter w % 4 (the only lanes it may
// access) with the 16x32bx2 shape, so its two half-warps take the two halves
// of one column unit for the same 16 starts (or, transposed, rows of B);
// split w / 4 takes every 4th unit.  Each start is thus served by 8 threads
// (4 splits x 2 halves).  Operands are stored in the canonical no-swizzle
// K-major layout: 8 rows x 16 bytes core matrices, K-adjacent core matrices
// 128 bytes apart (LBO), 8-row groups (K/8) * 128 bytes apart (SBO).
//
// The Adam epilogue is limited by the integer/logic pipe more than by TMEM
// latency: sign tests and rounding trackers are written as saturating
// multiplies, sums and one maximum per unit, which the FMA pipe takes
// (measured 5 % faster per launch than compares and selects), while issuing
// the next unit's TMEM loads ahead of the current unit's arithmetic measured
// slower.
//
// Every wait on the MMA barrier is bounded; on time-out the CTA records flag
// 16, leaves the loop together (block-wide vote), frees its TMEM and returns.
#include "common.cuh"
#include "extract_internal.cuh"
#include "tc_ptx.cuh"

#include <cuda_bf16.h>
#include <algorithm>
#include <type_traits>
#include <cmath>
#include <memory>
#include <vector>

namespace {

constexpr int kTileM = 64;
constexpr int kWarps = 16;
constexpr int kThreads = kWarps * 32;
constexpr int kSplits = kWarps / 4;
constexpr int kParts = kSplits * 2;  // threads per start
constexpr int kColD2 = 256;  // D2 when the accumulators cannot all have their own columns
constexpr int kIssuer = 32 * (kWarps - 4);  // issues every MMA: lane 0 of warp 12
constexpr int kTmemCols = 512;
constexpr int kNoNz = 0x7fffffff;

using namespace mape_tc;

// MN-major no-swizzle canonical layout ((T,1,m),(8,k)):((1,T,SBO),(1T,LBO)):
// the 8-row K groups are LBO apart and the 16-byte MN groups SBO apart.
#ifndef MAPE_TC_MN_LBO_IS_K
#define MAPE_TC_MN_LBO_IS_K 1
#endif
constexpr bool kMnLbo = MAPE_TC_MN_LBO_IS_K != 0;

// byte offset of element (row r, column k) in a no-swizzle K-major tile with K columns
__device__ __forceinline__ uint32_t op_off(int r, int k, int K) {
  return (uint32_t)((((r >> 3) * (K >> 3) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

// 8 bf16 (columns k0..k0+7, k0 a multiple of 8) of row r: one 16-byte store
__device__ __forceinline__ void store_row8(uint8_t* tile, int r, int k0, int K, const uint32_t (&w)[4]) {
  *reinterpret_cast<uint4*>(tile + op_off(r, k0, K)) = make_uint4(w[0], w[1], w[2], w[3]);
}
// W bf16 (W = 8 or 4; k0 a multiple of W) of row r
template <int W>
__device__ __forceinline__ void store_roww(uint8_t* tile, int r, int k0, int K, const uint32_t (&w)[W / 2]) {
  if constexpr (W == 8) *reinterpret_cast<uint4*>(tile + op_off(r, k0, K)) = make_uint4(w[0], w[1], w[2], w[3]);
  else *reinterpret_cast<uint2*>(tile + op_off(r, k0, K)) = make_uint2(w[0], w[1]);
}
template <int W>
using Width = std::integral_constant<int, W>;

// sign as a float: +-1, and 0 for 0 (and NaN)
__device__ __forceinline__ float sgn1(float x) { return fabsf(x) > 0.f ? copysignf(1.f, x) : 0.f; }

// the same sign from the FMA pipe instead of a compare and a select: |x|
// 2^75 2^75 saturated to [0, 1] (two exact scalings, so that a subnormal x
// also reaches 1; NaN gives 0) with the sign of x copied onto it, so that
// zero and NaN give a signed zero
__device__ __forceinline__ float sgn_sat(float x) {
  const float t = fabsf(x) * 0x1p75f;
  float a;
  asm("mul.sat.f32 %0, %1, %2;" : "=f"(a) : "f"(t), "f"(0x1p75f));
  return copysignf(a, x);
}

// bf16 pair {sign(a), sign(b)} (low half a): 0x3f80 = 1, 0xbf80 = -1, a signed
// zero (0x0000 or 0x8000) for zero and NaN
__device__ __forceinline__ uint32_t sign_bf16x2(float a, float b) {
  return pack_bf16x2(sgn_sat(a), sgn_sat(b));
}

// d/dz of the integrality term (ceil z - z)(z - floor z) of Eq. (3):
// ceil z + floor z - 2 z, which with e = z - rint(z) is sign(e) - 2 e (0 at
// the integers, +-1 - 2 e between them); every step is exact in FP32
__device__ __forceinline__ float frac_grad(float z, float rz) {
  const float e = z - rz;
  return fmaf(-2.f, e, sgn_sat(e));
}

// square root and reciprocal of the Adam denominator (v >= 0, den >= eps > 0)
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

struct TcParams {
  const int32_t* B;
  const int32_t* span;
  float* Zt;
  float* Mt;
  float* Vt;
  const float2* bias;  // (lr / (1 - beta1^t), 1 / sqrt(1 - beta2^t)) per step of this call
  int n, d, P, n_pad, d_pad;  // n_pad: rows of B in the MMA tile, padded to 16
  int span_pad;               // entries of the span table, pad16(n)
  int t0, T, period;
  float lambda1, lambda2, lr, eps, beta1, beta2, omb1, omb2;
  int nterms;   // 1: hi only, 2: hi + lo
  int use_bb;   // 1: transposed copy of B for the gradient MMA, 0: MN-major view
  int8_t* cand;
  int ldc;
  int64_t cap;
  unsigned long long* count;
  int32_t* flags;
  float* dbg_phi;
  float* dbg_grad;
};

struct Smem {  // byte offsets into dynamic shared memory
  uint32_t bf, bb, opa, opa2, ss, span, pz, pk, pl1, pfr, fl, fnz, slot, misc, bar, tmem, total;
};

// Transposed forward product, for tiles of at most 64 rows of B: one MMA
// chain D^T = B_tile . [hi(Z); lo(Z); round(Z)]^T (M = 64 rows of B, N = 64
// starts per operand, K = d) gives B hi(z), B lo(z) and B round(z) of every
// start in 10 instructions for d = 160 instead of 30 (an MMA instruction
// costs about the same whatever its M and N).
__host__ __device__ inline bool tc_transposed(int n_pad) { return n_pad <= 64; }

// per-start flag word bits
constexpr uint32_t kChanged = 1;    // rounding changed since the last collection
constexpr uint32_t kUnexact = 2;    // |round z| > 256 since the last collection
constexpr uint32_t kOutOfBox = 4;   // the current candidate fails C4 (rows in the MMA tile)
constexpr uint32_t kOutId = 8;      // ... fails C4 on the identity rows (identity-topped B)

__host__ __device__ inline uint32_t al(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

// Operand area: [hi | lo] of bf16(z) (nterms tiles of 64 x d_pad), then
// bf16(round z) (64 x d_pad).  S (64 starts x n_pad) overwrites the [hi | lo]
// tiles, or, in the transposed form, has its own MN-major tile (so that the
// three z tiles stay one N = 192 operand and are never overwritten).
__host__ __device__ inline Smem smem_layout(int n_pad, int d_pad, int nterms, int use_bb, int span_pad) {
  Smem s{};
  const bool tr = tc_transposed(n_pad);
  const uint32_t bf_rows = tr ? (uint32_t)kTileM : (uint32_t)n_pad;
  uint32_t o = 0;
  s.bf = o;   o = al(o + bf_rows * d_pad * 2, 1024);
  s.bb = o;   if (use_bb) o = al(o + (uint32_t)n_pad * d_pad * 2, 1024);
  s.opa = o;
  uint32_t zs = (uint32_t)nterms * d_pad > (uint32_t)n_pad ? (uint32_t)nterms * d_pad : (uint32_t)n_pad;
  if (tr) zs = (uint32_t)nterms * d_pad;
  s.opa2 = o + (uint32_t)kTileM * zs * 2;
  o = al(s.opa2 + (uint32_t)kTileM * d_pad * 2, 1024);
  s.ss = o;   if (tr) o = al(o + (uint32_t)kTileM * 64 * 2, 128);
  s.span = o; o = al(o + (uint32_t)span_pad * 4, 128);
  s.pz = o;   o = al(o + kParts * kTileM * 4, 128);
  s.pk = o;   o = al(o + kParts * kTileM * 4, 128);
  s.pl1 = o;  o = al(o + kParts * kTileM * 4, 128);
  s.pfr = o;  o = al(o + kParts * kTileM * 4, 128);
  s.fl = o;   o = al(o + kTileM * 4, 128);
  s.fnz = o;  o = al(o + kTileM * 4, 128);
  s.slot = o; o = al(o + kTileM * 8, 128);
  s.misc = o; o = al(o + 16 * 4 + 16, 16);  // out-of-box masks of the transposed test (one per warp), any-slot flag
  s.bar = o;  o = al(o + 32, 16);  // mbarriers: gradient, B round(z), forward, drain
  s.tmem = o; o = al(o + 4, 16);
  s.total = o;
  return s;
}

// kId: B = [I_d ; B'] (the basis of A = [C | I_m] is [I ; -C]).  The MMA tile
// then holds only B' (rows d .. n-1); the identity rows give (Bz)_j = z_j
// exactly, so their sign, bound test and the first nonzero entry of
// g = [round z ; B' round z] come from the FP32 master z in the Adam epilogue.
// kRes: z, m, v live in TMEM lanes 16-31 for the whole launch.
template <bool kId, bool kRes>
__device__ __forceinline__ void extract_tc_body(const TcParams& p, const int tile) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const Smem L = smem_layout(p.n_pad, p.d_pad, p.nterms, p.use_bb, p.span_pad);
  uint8_t* Bf = smem + L.bf;
  uint8_t* Bb = smem + L.bb;
  uint8_t* A1 = smem + L.opa;                           // hi(z)
  uint8_t* A1lo = smem + L.opa + kTileM * p.d_pad * 2;  // lo(z)
  uint8_t* A2 = smem + L.opa2;                          // round(z)
  uint8_t* Sop = smem + L.opa;                          // S, K-major (not transposed)
  uint8_t* sS = smem + L.ss;                            // S, MN-major (transposed)
  // transposed test: warp (quarter q, split k) writes the out-of-box bits of
  // starts 16 k .. 16 k + 15 over the rows of quarter q to slot 4 q + k
  uint32_t* s_outw = reinterpret_cast<uint32_t*>(smem + L.misc);
  int* s_any = reinterpret_cast<int*>(smem + L.misc + 16 * 4);
  float* s_span = reinterpret_cast<float*>(smem + L.span);  // box spans u - l, exact in FP32
  float* s_pz = reinterpret_cast<float*>(smem + L.pz);
  int32_t* s_pk = reinterpret_cast<int32_t*>(smem + L.pk);
  float* s_pl1 = reinterpret_cast<float*>(smem + L.pl1);
  float* s_pfr = reinterpret_cast<float*>(smem + L.pfr);
  uint32_t* s_fl = reinterpret_cast<uint32_t*>(smem + L.fl);
  int32_t* s_fnz = reinterpret_cast<int32_t*>(smem + L.fnz);
  long long* s_slot = reinterpret_cast<long long*>(smem + L.slot);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + L.tmem);
  const uint32_t bar = smem_u32(smem + L.bar);
  __shared__ int s_bad;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3, split = warp >> 2, half = lane >> 4;
  const int part = split * 2 + half;                      // which of the 8 threads of a start
  const int r = quarter * 16 + (lane & 15);               // start row in the tile
  const int64_t pg = (int64_t)tile * kTileM + r;          // global start
  const bool active = pg < p.P;
  const int n = p.n, d = p.d, n_pad = p.n_pad, d_pad = p.d_pad;
  const int nch = n_pad / 16, dch = d_pad / 16;
  const int r0 = kId ? d : 0;  // row of B held in row 0 of the MMA tile
  const int hoff = 8 * half;   // column offset of this half-warp inside a 16-column chunk
  const bool tr = tc_transposed(n_pad);
  const int bf_rows = tr ? kTileM : n_pad;  // the transposed form's M is 64 rows of B

  // ---- set-up: B in both operand layouts, span, flags ----
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int e = tid; e < bf_rows * d_pad; e += kThreads) {
    int i = e / d_pad, j = e % d_pad;
    int v = (i < n_pad && r0 + i < n && j < d) ? p.B[(int64_t)(r0 + i) * d + j] : 0;
    if (v > 256 || v < -256) s_bad = 1;
    __nv_bfloat16 hb = __float2bfloat16_rn((float)v);
    const uint16_t h = *reinterpret_cast<const uint16_t*>(&hb);
    *reinterpret_cast<uint16_t*>(Bf + op_off(i, j, d_pad)) = h;                              // N = rows, K = d
    if (p.use_bb && i < n_pad) *reinterpret_cast<uint16_t*>(Bb + op_off(j, i, n_pad)) = h;  // N = d, K = rows
  }
  for (int i = tid; i < p.span_pad; i += kThreads) s_span[i] = i < n ? (float)p.span[i] : 0.f;
  if (tid < kTileM) {
    s_fl[tid] = kChanged;  // the first collection of a call always counts
    s_fnz[tid] = kNoNz;
  }
  if (tid < 16) s_outw[tid] = 0u;
  if (tid == 0) *s_any = 0;
  if (tid == 0) {
    for (int b = 0; b < 4; ++b) mbar_init(bar + 8 * b, 1);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
  // upper 16 lanes of the quarter: this thread's start, columns z | m | v
  const uint32_t st_off = (uint32_t)(quarter * 32 + 16) << 16;
  const uint32_t col_m = (uint32_t)p.d_pad, col_v = 2u * (uint32_t)p.d_pad;
  bool bail = s_bad != 0;
  if (bail && tid == 0) atomicOr(p.flags, 8);

  // Accumulator columns (TMEM lanes 0-15 of each quarter).  Transposed form:
  // D^T = [B hi(z) | B lo(z) | B round(z)] in 64-column blocks from column 0
  // (lanes: rows of B), G from column 64 (nterms + 1) rounded up to 32, so
  // that the gradient MMA does not overwrite B round(z) while the candidate
  // is written.  Otherwise D1 (n_pad columns) and G share column 0 and D2 is
  // at column 256.  Every MMA of the CTA is issued by one thread.  (Issuing
  // the next step's forward MMAs during the Adam epilogue, as its operand
  // chunks are written, measured slower: MMAs running beside the epilogue
  // slow its TMEM traffic by more than they save.)
  const uint32_t colG_ = tr ? al(64u * (uint32_t)(p.nterms + 1), 32) : 0u;
  const uint32_t colD2 = tr ? 64u * (uint32_t)p.nterms : (uint32_t)kColD2;
  const bool issuer = tid == kIssuer;
  const uint32_t barG = bar, bar2 = bar + 8, barF = bar + 16, barD = bar + 24;
  // Column units of the initial pass and the epilogue, split u % 4 taking
  // unit u: 16 columns (8 per half-warp) for the rounds of four chunks; a last
  // round of fewer than four chunks is cut into units of 8 columns (4 per
  // half-warp), so that every split gets a share of it (with d_pad = 160 each
  // thread has 20 coordinates instead of 24 or 16).  Unit u covers columns
  // [ub, ub + 16) or [ub, ub + 8); the thread's own columns start at ub + W half.
  const int n_rounds = (dch + kSplits - 1) / kSplits;
  const int last_chunks = dch - kSplits * (n_rounds - 1);
  const int nu16 = last_chunks < kSplits ? kSplits * (n_rounds - 1) : dch;
  const int nu = last_chunks < kSplits ? nu16 + 2 * last_chunks : nu16;
  // A row's largest |z_j| is tracked per W-column group (the thread's columns
  // of one unit); the group bases are the same in every pass, so the group
  // holding the first maximiser is found again in the next epilogue.

  // FP32 master state of this thread's start: blocked [tile][d_pad/4][64][4],
  // four consecutive coordinates per 16-byte access, coalesced over 16 starts
  float4* const zb = reinterpret_cast<float4*>(p.Zt) + (size_t)tile * (d_pad / 4) * kTileM + r;
  float4* const mb = reinterpret_cast<float4*>(p.Mt) + (size_t)tile * (d_pad / 4) * kTileM + r;
  float4* const vb = reinterpret_cast<float4*>(p.Vt) + (size_t)tile * (d_pad / 4) * kTileM + r;

  const bool state_loaded = !bail;  // kRes: z, m, v are in TMEM from here on
  // ---- initial operand: bf16(z0) and the partial ||z0||_inf ----
  // Each thread keeps the largest |z_j| over its coordinates and the first of
  // its 8-column groups that holds it; padding coordinates and inactive starts
  // are 0 and never beat a real coordinate.
  float zinf_part = 0.f;
  int kmax_part = kNoNz;
  const uint32_t sbo_d = (uint32_t)(d_pad / 8) * 128, sbo_n = (uint32_t)(n_pad / 8) * 128;
  const uint32_t idesc_fwd = idesc_bf16(kTileM, n_pad);
  // forward MMAs (hi, then lo) of K-chunks [k0, k1) into D1 and B round(z)
  // MMAs of the same chunks into D2; D1 and D2 are overwritten by chunk 0
  auto issue_chunks = [&](int k0, int k1, bool fwd, bool d2) {
    if (tr) {  // one chain: A = the tile of B (M = 64), B = the z operand tiles (N = 64 per tile)
      const int nb = (fwd ? p.nterms : 0) + (d2 ? 1 : 0);
      if (nb == 0) return;
      const uint32_t bstart = smem_u32(fwd ? A1 : A2);
      const uint32_t idesc = idesc_bf16(kTileM, 64 * nb);
      const uint32_t dcol = fwd ? 0u : colD2;
      for (int kk = k0; kk < k1; ++kk) {
        const uint64_t a = make_desc(smem_u32(Bf) + kk * 256, 128, sbo_d);
        const uint64_t b = make_desc(bstart + kk * 256, 128, sbo_d);
        mma_bf16(tmem + dcol, a, b, idesc, kk > 0 ? 1u : 0u);
      }
      return;
    }
    if (fwd) {
      for (int term = 0; term < p.nterms; ++term) {
        const uint32_t abase = smem_u32(term == 0 ? A1 : A1lo);
        for (int kk = k0; kk < k1; ++kk) {
          const uint64_t a = make_desc(abase + kk * 256, 128, sbo_d);
          const uint64_t b = make_desc(smem_u32(Bf) + kk * 256, 128, sbo_d);
          mma_bf16(tmem, a, b, idesc_fwd, (term > 0 || kk > 0) ? 1u : 0u);
        }
      }
    }
    if (d2) {
      for (int kk = k0; kk < k1; ++kk) {
        const uint64_t a = make_desc(smem_u32(A2) + kk * 256, 128, sbo_d);
        const uint64_t b = make_desc(smem_u32(Bf) + kk * 256, 128, sbo_d);
        mma_bf16(tmem + colD2, a, b, idesc_fwd, kk > 0 ? 1u : 0u);
      }
    }
  };
  auto init_unit = [&](auto Wc, int ub) {
    constexpr int W = decltype(Wc)::value;
    const int c0 = ub + W * half;
    float zc[W];
#pragma unroll
    for (int k = 0; k < W / 4; ++k) {
      const float4 qz = zb[(c0 / 4 + k) * kTileM];
      zc[4 * k] = qz.x; zc[4 * k + 1] = qz.y; zc[4 * k + 2] = qz.z; zc[4 * k + 3] = qz.w;
    }
    if (kRes) {
      uint32_t wz[W], wm[W], wv[W];
#pragma unroll
      for (int k = 0; k < W / 4; ++k) {
        const float4 qm = mb[(c0 / 4 + k) * kTileM], qv = vb[(c0 / 4 + k) * kTileM];
        wm[4 * k] = __float_as_uint(qm.x); wm[4 * k + 1] = __float_as_uint(qm.y);
        wm[4 * k + 2] = __float_as_uint(qm.z); wm[4 * k + 3] = __float_as_uint(qm.w);
        wv[4 * k] = __float_as_uint(qv.x); wv[4 * k + 1] = __float_as_uint(qv.y);
        wv[4 * k + 2] = __float_as_uint(qv.z); wv[4 * k + 3] = __float_as_uint(qv.w);
      }
#pragma unroll
      for (int c = 0; c < W; ++c) wz[c] = __float_as_uint(zc[c]);
      tmem_stw<W>(tmem + st_off + ub, wz);
      tmem_stw<W>(tmem + st_off + col_m + ub, wm);
      tmem_stw<W>(tmem + st_off + col_v + ub, wv);
    }
    uint32_t wh[W / 2], wl[W / 2];
#pragma unroll
    for (int c = 0; c < W; c += 2) {
      wh[c >> 1] = pack_bf16x2(zc[c], zc[c + 1]);
      const __nv_bfloat162 hh = *reinterpret_cast<const __nv_bfloat162*>(&wh[c >> 1]);
      const float2 hf = __bfloat1622float2(hh);
      wl[c >> 1] = pack_bf16x2(zc[c] - hf.x, zc[c + 1] - hf.y);
    }
    float cmax = fabsf(zc[0]);
#pragma unroll
    for (int c = 1; c < W; ++c) cmax = fmaxf(cmax, fabsf(zc[c]));
    if (kmax_part == kNoNz || cmax > zinf_part) { zinf_part = cmax; kmax_part = c0; }
    store_roww<W>(A1, r, c0, d_pad, wh);
    if (p.nterms > 1) store_roww<W>(A1lo, r, c0, d_pad, wl);
  };
  for (int u = split; u < nu && !bail; u += kSplits) {
    if (u < nu16) init_unit(Width<8>{}, 16 * u);
    else init_unit(Width<4>{}, 16 * nu16 + 8 * (u - nu16));
  }
  s_pz[part * kTileM + r] = zinf_part;
  s_pk[part * kTileM + r] = kmax_part;
  if (kRes) tc_wait_st();
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  const bool dbg_on = (p.dbg_phi != nullptr || p.dbg_grad != nullptr);
  // gradient MMA: B operand K-major from the transposed copy, or MN-major
  // (bit 16) straight from the forward tile; A = S MN-major (bit 15) in the
  // transposed form
  const uint32_t idesc_bwd = idesc_bf16(kTileM, d_pad) | (p.use_bb ? 0u : (1u << 16)) | (tr ? (1u << 15) : 0u);

  // combine the partials of ||z||_inf: max, ties to the lower group, so that
  // kmax is the 8-column group holding the first maximiser of |z|
  auto combine_zinf = [&](float& zinf, int& kmax) {
    zinf = 0.f;
    kmax = kNoNz;
    for (int s = 0; s < kParts; ++s) {
      float z = s_pz[s * kTileM + r];
      int k = s_pk[s * kTileM + r];
      if (k == kNoNz) continue;
      if (kmax == kNoNz || z > zinf || (z == zinf && k < kmax)) { zinf = z; kmax = k; }
    }
  };
  float zinf;
  int kmax;
  combine_zinf(zinf, kmax);

  // tests the candidate held in D2 (bound test, first nonzero entry) ...
  // transposed form: v holds B round(z) of row i of B (lane) for the 8 starts
  // 16 split + hoff + c (columns), loaded with the sign phase's operands;
  // every lane calls this (warp-collective reductions)
  auto test_candidate_tr = [&](const uint32_t (&v)[8]) {
      uint32_t outm = 0;  // bit 8 half + c: that start fails C4 on row i
      int key[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) key[c] = kNoNz;
      if (quarter < nch) {  // warp-uniform: the quarter holds rows of the tile
        const int i = r0 + quarter * 16 + (lane & 15);
        if (i < n) {
          const float sp = s_span[i];
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const float g = __uint_as_float(v[c]);  // an integer, exact
            if (fabsf(g) > sp) outm |= 1u << (8 * half + c);
            if (!kId && g != 0.f) key[c] = (i << 1) | (g < 0.f ? 1 : 0);
          }
        }
      }
      outm = __reduce_or_sync(0xffffffffu, outm);
      if (lane == 0) s_outw[quarter * 4 + split] = outm;  // every warp writes its slot on every test
      if (!kId) {  // first nonzero row: minimum over the 16 rows of the half-warp
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          int k = key[c];
#pragma unroll
          for (int o = 1; o < 16; o <<= 1) k = min(k, __shfl_xor_sync(0xffffffffu, k, o));
          if ((lane & 15) == 0 && k != kNoNz) atomicMin(&s_fnz[16 * split + hoff + c], k);
        }
      }
  };
  auto test_candidate = [&]() {
    int first = kNoNz;
    bool out = false;
    for (int ch = split; ch < nch; ch += kSplits) {
      uint32_t v[8];
      tmem_ld8x2(tmem + lane_off + colD2 + ch * 16, v);
      tc_wait_ld();
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int i = r0 + ch * 16 + hoff + c;  // row of B
        const float g = __uint_as_float(v[c]);  // an integer, exact
        if (i < n) {
          out |= fabsf(g) > s_span[i];
          if (!kId && g != 0.f && (i << 1) < first) first = (i << 1) | (g < 0.f ? 1 : 0);
        }
      }
    }
    if (out) atomicOr(&s_fl[r], kOutOfBox);
    if (!kId && first != kNoNz) atomicMin(&s_fnz[r], first);
  };
  // ... and appends it in canonical sign (needs a barrier between the two).
  // decide_slot leaves the slot and the sign in s_slot (2 slot + [negative],
  // -1 for none) and clears the start's collection state; s_any was cleared
  // before the barrier that precedes it.
  auto decide_slot = [&]() {
    if (part != 0) return;
    long long slot = -1;
    uint32_t f = s_fl[r];
    if (tr) {
      const int k = r >> 4, b = r & 15;
      if (((s_outw[k] | s_outw[4 + k] | s_outw[8 + k] | s_outw[12 + k]) >> b) & 1u) f |= kOutOfBox;
    }
    int fnz = s_fnz[r];
    if (active && (f & kChanged) && !(f & (kOutOfBox | kOutId)) && fnz != kNoNz) {
      if (f & kUnexact) {
        atomicOr(p.flags, 2);
      } else {
        unsigned long long at = atomicAdd(p.count, 1ull);
        if ((int64_t)at < p.cap) slot = (long long)at;
        else atomicOr(p.flags, 1);
      }
    }
    s_slot[r] = slot >= 0 ? (slot << 1) | (fnz & 1) : -1;
    if (slot >= 0) *s_any = 1;
    s_fl[r] = 0;
    s_fnz[r] = kNoNz;
  };
  // every lane of the warp executes the (warp-collective) TMEM loads; only
  // lanes whose start has a slot store.  In the transposed form the rows of
  // the tile come from vd, the B round(z) words the sign phase loaded for the
  // candidate test: a TMEM load here would run beside the gradient MMA, and
  // the two slow each other down.
  auto write_candidate = [&](const uint32_t (&vd)[8]) {
    if (*s_any == 0) return;  // CTA-uniform: no start of the tile has a slot
    const long long sv = s_slot[r];
    const long long slot = sv >= 0 ? sv >> 1 : -1;
    const int sgn = (sv & 1) ? -1 : 1;
    int8_t* row = slot >= 0 ? p.cand + slot * p.ldc : nullptr;
    if (kId) {
      // identity rows: g_j = round z_j, held as BF16 in the round(z) operand tile
      for (int ch = split; ch < dch && row; ch += kSplits) {
        const int c0 = ch * 16 + hoff;
        const uint4 q = *reinterpret_cast<const uint4*>(A2 + op_off(r, c0, d_pad));
        const uint32_t wv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int j = c0 + c;
          const float zr = __uint_as_float((c & 1) ? (wv[c >> 1] & 0xffff0000u) : (wv[c >> 1] << 16));
          if (j < d) row[j] = (int8_t)(sgn * __float2int_rn(zr));
        }
      }
    }
    if (tr) {
      // rows of the tile from D2^T: this thread holds row i of B for the 8
      // starts 16 split + hoff + c
      if (quarter < nch) {
        const int i = r0 + quarter * 16 + (lane & 15);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int rs = 16 * split + hoff + c;
          const long long sv = s_slot[rs];
          if (sv >= 0 && i < n) {
            const int sg = (sv & 1) ? -1 : 1;
            p.cand[(sv >> 1) * p.ldc + i] = (int8_t)(sg * __float2int_rn(__uint_as_float(vd[c])));
          }
        }
      }
      if (row && part == 0)
        for (int b = n; b < p.ldc; ++b) row[b] = 0;
      return;
    }
    if (kId) {
      // rows of B' from D2 (warp-collective loads: every lane executes them)
      for (int ch = split; ch < nch; ch += kSplits) {
        uint32_t v[8];
        tmem_ld8x2(tmem + lane_off + colD2 + ch * 16, v);
        tc_wait_ld();
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int i = r0 + ch * 16 + hoff + c;
          if (row && i < n) row[i] = (int8_t)(sgn * __float2int_rn(__uint_as_float(v[c])));
        }
      }
      if (row && part == 0)
        for (int b = n; b < p.ldc; ++b) row[b] = 0;
    } else {
      for (int ch = split; ch < nch; ch += kSplits) {
        uint32_t v[8];
        tmem_ld8x2(tmem + lane_off + colD2 + ch * 16, v);
        tc_wait_ld();
        uint32_t w[2] = {0, 0};
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          int g = sgn * __float2int_rn(__uint_as_float(v[c]));
          w[c >> 2] |= ((uint32_t)(g & 0xff)) << ((c & 3) * 8);
        }
        if (row) *reinterpret_cast<uint2*>(row + ch * 16 + hoff) = make_uint2(w[0], w[1]);
      }
      if (row && part == 0)
        for (int off = n_pad; off < p.ldc; off += 16) *reinterpret_cast<uint4*>(row + off) = make_uint4(0, 0, 0, 0);
    }
  };
  uint32_t phaseG = 0, phaseF = 0, phase2 = 0;
  // gradient MMA wait; a time-out anywhere ends the launch for the whole CTA
  auto wait_grad = [&]() -> bool {
    const bool ok = mbar_wait_bounded(barG, phaseG);
    phaseG ^= 1;
    const bool any_bad = __syncthreads_or(!ok) != 0;
    if (any_bad && tid == 0) atomicOr(p.flags, 16);
    tc_fence_after();
    return !any_bad;
  };

  for (int s = 0; s < p.T && !bail; ++s) {
    const int t = p.t0 + s + 1;              // global step number
    const bool collect_prev = s >= 1 && ((t - 1) % p.period == 0);
    const bool dbg_step = dbg_on && s == 0;
    // (1) forward MMAs (and B round(z) of the previous step's candidate)
    if (issuer) {
      tc_fence_after();
      issue_chunks(0, dch, true, tr && collect_prev);  // transposed: one chain
      mma_commit(barF);
      if (!tr && collect_prev) {
        issue_chunks(0, dch, false, true);
        mma_commit(bar2);
      }
    }
    // ||z||_inf and the group of its first maximiser, from the partials the
    // last epilogue left (the forward chain is already on its way)
    if (s > 0) combine_zinf(zinf, kmax);
    // every thread waits itself; the time-out vote joins the barrier after
    // the sign phase (warp-uniform: the TMEM loads are collective)
    bool late = __any_sync(0xffffffffu, !mbar_wait_bounded(barF, phaseF));
    phaseF ^= 1;
    tc_fence_after();
    // (2) S = sign(D1) into shared memory; test the previous step's candidate
    float l1 = 0.f;
    uint32_t vd[8];  // transposed form: B round(z) of the previous step's candidate
    if (tr) {
      // this thread: row i of the tile (lane), starts 16 split + hoff + c
      // (columns); B z = B hi(z) + B lo(z)
      float y[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) y[c] = 0.f;
      if (quarter < nch) {  // warp-uniform: the quarter holds rows of the tile
        uint32_t vh[8], vl[8];
        tmem_ld8x2(tmem + lane_off + 16 * split, vh);
        if (p.nterms > 1) tmem_ld8x2(tmem + lane_off + 64 + 16 * split, vl);
        if (collect_prev) tmem_ld8x2(tmem + lane_off + colD2 + 16 * split, vd);
        tc_wait_ld();
#pragma unroll
        for (int c = 0; c < 8; ++c)
          y[c] = p.nterms > 1 ? __uint_as_float(vh[c]) + __uint_as_float(vl[c]) : __uint_as_float(vh[c]);
        uint32_t w[4];
#pragma unroll
        for (int c = 0; c < 8; c += 2) w[c >> 1] = sign_bf16x2(y[c], y[c + 1]);
        // MN-major S: element (start rs, row i) at (i / 8) 1024 + (rs / 8) 128 + (i % 8) 16 + (rs % 8) 2
        const int i = quarter * 16 + (lane & 15), rs = 16 * split + hoff;
        *reinterpret_cast<uint4*>(sS + (i >> 3) * 1024 + (rs >> 3) * 128 + (i & 7) * 16) =
            make_uint4(w[0], w[1], w[2], w[3]);
      }
      if (dbg_step) {  // l1 of the tile rows per start: parts 0-3 are the quarters' row sums
        float a[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          a[c] = fabsf(y[c]);
#pragma unroll
          for (int o = 1; o < 16; o <<= 1) a[c] += __shfl_xor_sync(0xffffffffu, a[c], o);
        }
        if ((lane & 15) == 0)
          for (int c = 0; c < 8; ++c) s_pl1[quarter * kTileM + 16 * split + hoff + c] = a[c];
        if ((lane & 15) == 1)
          for (int c = 0; c < 8; ++c) s_pl1[(quarter + 4) * kTileM + 16 * split + hoff + c] = 0.f;
      }
      if (collect_prev) test_candidate_tr(vd);
    }
    for (int ch = split; ch < nch && !tr; ch += kSplits) {
      uint32_t v[8];
      tmem_ld8x2(tmem + lane_off + ch * 16, v);
      tc_wait_ld();
      uint32_t w[4];
#pragma unroll
      for (int c = 0; c < 8; c += 2) w[c >> 1] = sign_bf16x2(__uint_as_float(v[c]), __uint_as_float(v[c + 1]));
      if (dbg_step) {
#pragma unroll
        for (int c = 0; c < 8; ++c) l1 += fabsf(__uint_as_float(v[c]));
      }
      store_row8(Sop, r, ch * 16 + hoff, n_pad, w);
    }
    if (dbg_step && !tr) s_pl1[part * kTileM + r] = l1;
    if (collect_prev && !tr) {  // transposed: D2 came with the forward chain, tested above
      late |= __any_sync(0xffffffffu, !mbar_wait_bounded(bar2, phase2));
      phase2 ^= 1;
      tc_fence_after();
      if (!late) test_candidate();
    }
    if (collect_prev && tid == 0) *s_any = 0;  // every thread read it in the last write_candidate
    tc_wait_ld();
    tc_fence_before();
    fence_async_smem();
    if (__syncthreads_or(late)) {
      if (tid == 0) atomicOr(p.flags, 16);
      bail = true;
      break;
    }
    // (3) gradient MMA, overlapped with appending the previous candidate
    if (issuer) {
      tc_fence_after();
      for (int kk = 0; kk < nch; ++kk) {
        // A = S: K-major, or MN-major (transposed form; K groups 1024 bytes
        // apart, 8-start groups 128 bytes apart)
        uint64_t a = tr ? make_desc(smem_u32(sS) + kk * 2048, kMnLbo ? 1024 : 128, kMnLbo ? 128 : 1024)
                        : make_desc(smem_u32(Sop) + kk * 256, 128, sbo_n);
        // K step kk covers rows 16kk..16kk+15 of B: two 8-row core-matrix groups
        uint64_t b = p.use_bb ? make_desc(smem_u32(Bb) + kk * 256, 128, sbo_n)
                              : make_desc(smem_u32(Bf) + kk * 2 * sbo_d, kMnLbo ? sbo_d : 128, kMnLbo ? 128 : sbo_d);
        mma_bf16(tmem + colG_, a, b, idesc_bwd, kk > 0);
      }
      mma_commit(barG);
    }
    if (collect_prev) {
      decide_slot();
      __syncthreads();
      write_candidate(vd);
    }
    if (kId && part == 0) {  // the Adam epilogue recomputes these for round(z) of this step
      s_fnz[r] = kNoNz;
      s_fl[r] &= ~kOutId;
    }
    if (!wait_grad()) { bail = true; break; }
    // (4) Adam on the FP32 master state; next operands
    // Adam in the form z -= (lr / bc1) m / (sqrt(v) / sqrt(bc2) + eps), with
    // lr / bc1 and 1 / sqrt(bc2) formed in double on the host
    const float2 ad = p.bias[s];
    const float step = ad.x, rsb2 = ad.y;
    // The inverse-norm term of Eq. (3), -lambda2 / ||z||_inf^2 times the sign
    // of z at the first maximiser of |z|, is nonzero only while
    // 0 < ||z||_inf < 1; kmax is the column group holding that maximiser.
    const bool inv_on = zinf < 1.f && zinf > 0.f;
    const float inv_term = inv_on ? -p.lambda2 / (zinf * zinf) : 0.f;
    // G (TMEM) and the master z, m, v of the W coordinates c0 .. c0+W-1 (unit base ub)
    auto load_state = [&](int ub, int c0, auto& v, auto& zc, auto& mc, auto& vc) {
      constexpr int W = std::extent<std::remove_reference_t<decltype(v)>>::value;
      tmem_ldw<W>(tmem + lane_off + colG_ + ub, v);  // completes under the loads below
      if (kRes) {
        uint32_t tz[W], tm[W], tv[W];
        tmem_ldw<W>(tmem + st_off + ub, tz);
        tmem_ldw<W>(tmem + st_off + col_m + ub, tm);
        tmem_ldw<W>(tmem + st_off + col_v + ub, tv);
        tc_wait_ld();
#pragma unroll
        for (int c = 0; c < W; ++c) {
          zc[c] = __uint_as_float(tz[c]);
          mc[c] = __uint_as_float(tm[c]);
          vc[c] = __uint_as_float(tv[c]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < W / 4; ++k) {
          const int g4 = c0 / 4 + k;
          const float4 qz = zb[g4 * kTileM], qm = mb[g4 * kTileM], qv = vb[g4 * kTileM];
          zc[4 * k] = qz.x; zc[4 * k + 1] = qz.y; zc[4 * k + 2] = qz.z; zc[4 * k + 3] = qz.w;
          mc[4 * k] = qm.x; mc[4 * k + 1] = qm.y; mc[4 * k + 2] = qm.z; mc[4 * k + 3] = qm.w;
          vc[4 * k] = qv.x; vc[4 * k + 1] = qv.y; vc[4 * k + 2] = qv.z; vc[4 * k + 3] = qv.w;
        }
        tc_wait_ld();
      }
    };
    // the gradient of Eq. (3) at coordinates c0 .. c0+W-1: G + lambda1 (ceil z
    // + floor z - 2 z), the inverse-norm term, and for identity-topped B the
    // identity rows' sign(z_j)
    auto unit_grad = [&](int c0, const auto& v, const auto& zc, const auto& rz, auto& g) {
      constexpr int W = std::extent<std::remove_reference_t<decltype(g)>>::value;
#pragma unroll
      for (int c = 0; c < W; ++c) g[c] = fmaf(p.lambda1, frac_grad(zc[c], rz[c]), __uint_as_float(v[c]));
      if (inv_on && c0 == kmax) {
        bool hit = false;
#pragma unroll
        for (int c = 0; c < W; ++c) {
          if (!hit && fabsf(zc[c]) == zinf) {
            g[c] += inv_term * sgn1(zc[c]);
            hit = true;
          }
        }
      }
      if (kId) {
#pragma unroll
        for (int c = 0; c < W; ++c) g[c] += sgn_sat(zc[c]);
      }
    };
    // debug outputs of the first step: the integrality sum of Phi, the l1 norm
    // of the identity rows and the gradient, before the state is overwritten
    float frac = 0.f, l1_id = 0.f;
    auto dbg_unit = [&](auto Wc, int ub) {
      constexpr int W = decltype(Wc)::value;
      const int c0 = ub + W * half;
      uint32_t v[W];
      float zc[W], mc[W], vc[W], rz[W], g[W];
      load_state(ub, c0, v, zc, mc, vc);
#pragma unroll
      for (int c = 0; c < W; ++c) rz[c] = rintf(zc[c]);
      unit_grad(c0, v, zc, rz, g);
#pragma unroll
      for (int c = 0; c < W; ++c) {
        const int j = c0 + c;
        if (!active || j >= d) continue;
        const float z = zc[c], fl = floorf(z);
        frac += (z - fl) * (ceilf(z) - z);
        if (kId) l1_id += fabsf(z);
        if (p.dbg_grad) p.dbg_grad[pg * d + j] = g[c];
      }
    };
    if (dbg_step) {
      for (int u = split; u < nu; u += kSplits) {
        if (u < nu16) dbg_unit(Width<8>{}, 16 * u);
        else dbg_unit(Width<4>{}, 16 * nu16 + 8 * (u - nu16));
      }
    }
    float nzinf = 0.f;
    int nkmax = kNoNz, first_id = kNoNz;
    bool changed = false, unexact = false, out_id = false;
    // rounding changes: the sum of |rint(z_new) - rint(z_old)| over the
    // thread's coordinates (integers, exactly summed; 0 iff none changed)
    float dsum = 0.f;
    auto epi_unit = [&](auto Wc, int ub) {
      constexpr int W = decltype(Wc)::value;
      const int c0 = ub + W * half;
      uint32_t v[W];
      float zc[W], mc[W], vc[W], rz[W], g[W];
      load_state(ub, c0, v, zc, mc, vc);
#pragma unroll
      for (int c = 0; c < W; ++c) rz[c] = rintf(zc[c]);
      unit_grad(c0, v, zc, rz, g);
      float zn[W], rn[W];
      uint32_t zo[W], mo[W], vo[W];
#pragma unroll
      for (int c = 0; c < W; ++c) {
        const float m = fmaf(p.beta1, mc[c], p.omb1 * g[c]);
        const float vv = fmaf(p.beta2, vc[c], p.omb2 * g[c] * g[c]);
        const float den = fmaf(sqrt_approx(vv), rsb2, p.eps);
        // padding coordinates (j >= d) have zero gradient and stay at 0
        zn[c] = fmaf(-step, m * rcp_approx(den), zc[c]);
        rn[c] = rintf(zn[c]);
        zo[c] = __float_as_uint(zn[c]);
        mo[c] = __float_as_uint(m);
        vo[c] = __float_as_uint(vv);
        // padding coordinates (z = 0 throughout) and inactive starts leave
        // every tracker unchanged: their roundings never change, are 0, are
        // within any box and never beat a real coordinate's |z| or index
        dsum += fabsf(rn[c] - rz[c]);
      }
      float cmax = fabsf(zn[0]);
#pragma unroll
      for (int c = 1; c < W; ++c) cmax = fmaxf(cmax, fabsf(zn[c]));
      if (nkmax == kNoNz || cmax > nzinf) { nzinf = cmax; nkmax = c0; }
      if (kId) {  // identity rows of g = B round(z): bound test and first nonzero entry
        float sp[W];
#pragma unroll
        for (int k = 0; k < W / 4; ++k) {
          const float4 q4 = *reinterpret_cast<const float4*>(s_span + c0 + 4 * k);
          sp[4 * k] = q4.x; sp[4 * k + 1] = q4.y; sp[4 * k + 2] = q4.z; sp[4 * k + 3] = q4.w;
        }
        const bool nz = cmax > 0.5f;  // some rint(z_j) != 0
#pragma unroll
        for (int c = 0; c < W; ++c) out_id |= fabsf(rn[c]) > sp[c];
        if (first_id == kNoNz && nz) {
#pragma unroll
          for (int c = 0; c < W; ++c)
            if (first_id == kNoNz && rn[c] != 0.f) first_id = ((c0 + c) << 1) | (rn[c] < 0.f ? 1 : 0);
        }
      }
      uint32_t w1[W / 2], wl[W / 2], w2[W / 2];
#pragma unroll
      for (int c = 0; c < W; c += 2) {
        w1[c >> 1] = pack_bf16x2(zn[c], zn[c + 1]);
        const float2 hf = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w1[c >> 1]));
        wl[c >> 1] = pack_bf16x2(zn[c] - hf.x, zn[c + 1] - hf.y);
        w2[c >> 1] = pack_bf16x2(rn[c], rn[c + 1]);
      }
      if (kRes) {
        tmem_stw<W>(tmem + st_off + ub, zo);
        tmem_stw<W>(tmem + st_off + col_m + ub, mo);
        tmem_stw<W>(tmem + st_off + col_v + ub, vo);
      } else {
#pragma unroll
        for (int k = 0; k < W / 4; ++k) {
          const int g4 = c0 / 4 + k;
          zb[g4 * kTileM] = make_float4(zn[4 * k], zn[4 * k + 1], zn[4 * k + 2], zn[4 * k + 3]);
          mb[g4 * kTileM] = make_float4(__uint_as_float(mo[4 * k]), __uint_as_float(mo[4 * k + 1]),
                                        __uint_as_float(mo[4 * k + 2]), __uint_as_float(mo[4 * k + 3]));
          vb[g4 * kTileM] = make_float4(__uint_as_float(vo[4 * k]), __uint_as_float(vo[4 * k + 1]),
                                        __uint_as_float(vo[4 * k + 2]), __uint_as_float(vo[4 * k + 3]));
        }
      }
      store_roww<W>(A1, r, c0, d_pad, w1);
      if (p.nterms > 1) store_roww<W>(A1lo, r, c0, d_pad, wl);
      store_roww<W>(A2, r, c0, d_pad, w2);
    };
    for (int u = split; u < nu; u += kSplits) {
      if (u < nu16) epi_unit(Width<8>{}, 16 * u);
      else epi_unit(Width<4>{}, 16 * nu16 + 8 * (u - nu16));
    }
    s_pz[part * kTileM + r] = nzinf;
    s_pk[part * kTileM + r] = nkmax;
    if (dbg_step) {
      s_pfr[part * kTileM + r] = frac;
      if (kId) s_pl1[part * kTileM + r] += l1_id;
    }
    changed = dsum != 0.f;
    // |rint(z_j)| > 256 for some j iff max |z_j| > 256.5 (256.5 rounds to 256)
    unexact = nzinf > 256.5f;
    uint32_t fbits = (changed ? kChanged : 0u) | (unexact ? kUnexact : 0u) | (out_id ? kOutId : 0u);
    if (fbits) atomicOr(&s_fl[r], fbits);
    if (kId && first_id != kNoNz) atomicMin(&s_fnz[r], first_id);
    tc_wait_ld();
    if (kRes) tc_wait_st();
    tc_fence_before();
    fence_async_smem();
    __syncthreads();
    if (dbg_step && part == 0 && active && p.dbg_phi) {
      float L1 = 0.f, FR = 0.f;
      for (int q = 0; q < kParts; ++q) { L1 += s_pl1[q * kTileM + r]; FR += s_pfr[q * kTileM + r]; }
      float inv = zinf > 0.f ? fmaxf(1.f / zinf - 1.f, 0.f) : INFINITY;
      p.dbg_phi[pg] = L1 + p.lambda1 * FR + p.lambda2 * inv;
    }
  }

  // the candidate of the last step
  if (!bail && p.T > 0 && ((p.t0 + p.T) % p.period == 0)) {
    if (issuer) {
      tc_fence_after();
      issue_chunks(0, dch, false, true);
      mma_commit(bar2);
    }
    bool late = __any_sync(0xffffffffu, !mbar_wait_bounded(bar2, phase2));
    phase2 ^= 1;
    tc_fence_after();
    uint32_t vd[8];
    if (tr) {
      if (quarter < nch && !late) {
        tmem_ld8x2(tmem + lane_off + colD2 + 16 * split, vd);
        tc_wait_ld();
      }
      if (!late) test_candidate_tr(vd);
    } else if (!late) {
      test_candidate();
    }
    if (tid == 0) *s_any = 0;
    tc_wait_ld();
    if (__syncthreads_or(late)) {
      if (tid == 0) atomicOr(p.flags, 16);
    } else {
      decide_slot();
      __syncthreads();
      write_candidate(vd);
    }
  }
  // arrives once every MMA of the CTA has completed (all were issued by this
  // thread); TMEM is freed only then, also after a time-out
  if (issuer) mma_commit(barD);
  if (kRes && state_loaded) {  // the state leaves TMEM for the caller's arrays
    for (int ch = split; ch < dch; ch += kSplits) {
      const int c0 = ch * 16 + hoff;
      uint32_t tz[8], tm[8], tv[8];
      tmem_ld8x2(tmem + st_off + ch * 16, tz);
      tmem_ld8x2(tmem + st_off + col_m + ch * 16, tm);
      tmem_ld8x2(tmem + st_off + col_v + ch * 16, tv);
      tc_wait_ld();
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int g4 = c0 / 4 + k;
        zb[g4 * kTileM] = make_float4(__uint_as_float(tz[4 * k]), __uint_as_float(tz[4 * k + 1]),
                                      __uint_as_float(tz[4 * k + 2]), __uint_as_float(tz[4 * k + 3]));
        mb[g4 * kTileM] = make_float4(__uint_as_float(tm[4 * k]), __uint_as_float(tm[4 * k + 1]),
                                      __uint_as_float(tm[4 * k + 2]), __uint_as_float(tm[4 * k + 3]));
        vb[g4 * kTileM] = make_float4(__uint_as_float(tv[4 * k]), __uint_as_float(tv[4 * k + 1]),
                                      __uint_as_float(tv[4 * k + 2]), __uint_as_float(tv[4 * k + 3]));
      }
    }
  }
  tc_wait_ld();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    mbar_wait_bounded(barD, 0);
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

template <bool kId, bool kRes>
__global__ void __launch_bounds__(kThreads, 1) extract_tc_kernel(TcParams p) {
  extract_tc_body<kId, kRes>(p, blockIdx.x);
}

// Many instances in one launch: CTA b runs tile work[b].y of instance
// work[b].x, whose parameters (own B, state, candidate buffer, steps) are
// table[work[b].x]; the dynamic shared memory is sized for the largest tile.
template <bool kId, bool kRes>
__global__ void __launch_bounds__(kThreads, 1) extract_tc_batch_kernel(const TcParams* __restrict__ table,
                                                                       const int2* __restrict__ work) {
  __shared__ TcParams s_p;
  const int2 w = work[blockIdx.x];
  if (threadIdx.x == 0) s_p = table[w.x];
  __syncthreads();
  extract_tc_body<kId, kRes>(s_p, w.y);
}

// [P x d] row-major  <->  blocked [ceil(P/64)][d_pad/4][64][4] (zero padded)
__global__ void pack_blocked_kernel(const float* __restrict__ in, float* __restrict__ out, int P, int d, int d_pad,
                                    int64_t total) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int c = (int)(e & 3);
  const int r = (int)((e >> 2) % kTileM);
  const int64_t g = e / (4 * kTileM);
  const int g4 = (int)(g % (d_pad / 4));
  const int64_t tile = g / (d_pad / 4);
  const int64_t row = tile * kTileM + r;
  const int j = g4 * 4 + c;
  out[e] = (row < P && j < d) ? in[row * d + j] : 0.f;
}

__global__ void unpack_blocked_kernel(const float* __restrict__ in, float* __restrict__ out, int P, int d, int d_pad) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)P * d) return;
  const int64_t row = e / d;
  const int j = (int)(e % d);
  const int64_t tile = row / kTileM;
  const int r = (int)(row % kTileM);
  out[e] = in[((tile * (d_pad / 4) + j / 4) * kTileM + r) * 4 + (j & 3)];
}

int pad16(int x) { return (x + 15) / 16 * 16; }

// flag = 1 unless the top d x d block of B is the identity
__global__ void identity_top_kernel(const int32_t* __restrict__ B, int d, int32_t* __restrict__ flag) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)d * d) return;
  int i = (int)(e / d), j = (int)(e % d);
  if (B[(int64_t)i * d + j] != (i == j ? 1 : 0)) atomicOr(flag, 1);
}

// rows of B held in the MMA tile: all n, or the n - d rows below the identity
int tile_rows(int n, int d, bool id) { return pad16(id ? (n - d > 0 ? n - d : 1) : n); }

}  // namespace

namespace mape_detail {

constexpr uint32_t kSmemLimit = 232448 - 2048;  // opt-in maximum less static shared memory

#ifndef MAPE_TC_FORCE_MN
#define MAPE_TC_FORCE_MN 0
#endif

// The transposed copy of B is used when it fits, else the MN-major view.
int tc_use_bb(int n_pad, int d_pad, int nterms, int span_pad) {
  if (MAPE_TC_FORCE_MN) return 0;
  return smem_layout(n_pad, d_pad, nterms, 1, span_pad).total <= kSmemLimit ? 1 : 0;
}

bool tc_fits(int32_t n, int32_t d, int nterms, bool id) {
  int n_pad = tile_rows(n, d, id), d_pad = pad16(d), span_pad = pad16(n);
  if (n_pad > 256 || d_pad > 256) return false;
  return smem_layout(n_pad, d_pad, nterms, tc_use_bb(n_pad, d_pad, nterms, span_pad), span_pad).total <= kSmemLimit;
}

// Supported when some B of this shape runs: identity-topped bases need the
// smaller tile; a general B of a shape only the identity-topped tile fits is
// refused with MAPE_ERR_SHAPE at launch.
bool extract_tc_supported(int32_t n, int32_t d, int32_t precision) {
  const int nterms = precision == MAPE_PREC_BF16X1 ? 1 : 2;
  return tc_fits(n, d, nterms, true) || tc_fits(n, d, nterms, false);
}

size_t extract_tc_workspace(int32_t n, int32_t d, int32_t P, int32_t precision) {
  if (!extract_tc_supported(n, d, precision)) return 0;
  Sizer s;
  const size_t blocked = (size_t)ceil_div(P, kTileM) * kTileM * pad16(d);
  for (int k = 0; k < 3; ++k) s.take<float>(blocked);  // z, m, v blocked (carved separately)
  s.take<float2>((size_t)1 << 20);  // bias-correction table, up to 2^20 steps per call
  s.take<int32_t>(1);               // identity-top flag
  return s.bytes();
}

// Carves one call's workspace, uploads its Adam bias table, packs its state
// into the blocked layout and fills its kernel parameters (no launch of the
// extraction itself, no synchronisation).
static int tc_prepare(const mape_extract_args* a, bool id, cudaStream_t st, TcParams& p, uint32_t& smem) {
  const int n = a->n, d = a->d, P = a->P;
  if (a->T > (1 << 20)) return MAPE_ERR_SHAPE;
  const int nterms = a->precision == MAPE_PREC_BF16X1 ? 1 : 2;
  if (!tc_fits(n, d, nterms, id)) return MAPE_ERR_SHAPE;
  Carver cv(a->workspace, a->workspace_bytes);
  const int d_pad = pad16(d);
  const int64_t blocked = ceil_div(P, kTileM) * kTileM * (int64_t)d_pad;
  float* Zt = cv.take<float>((size_t)blocked);
  float* Mt = cv.take<float>((size_t)blocked);
  float* Vt = cv.take<float>((size_t)blocked);
  float2* bias = cv.take<float2>((size_t)1 << 20);
  cv.take<int32_t>(1);
  if (!cv.ok) return MAPE_ERR_CAPACITY;
  std::vector<float2> bc((size_t)a->T);
  for (int s = 0; s < a->T; ++s) {
    double t = (double)a->t0 + s + 1;
    double bc1 = 1.0 - std::pow(a->beta1, t), bc2 = 1.0 - std::pow(a->beta2, t);
    bc[s] = make_float2((float)((double)a->lr / bc1), (float)(1.0 / std::sqrt(bc2)));
  }
  MAPE_CUDA_TRY(cudaMemcpyAsync(bias, bc.data(), sizeof(float2) * bc.size(), cudaMemcpyHostToDevice, st));
  const unsigned gpack = (unsigned)ceil_div(blocked, 256);
  mape_detail::launch(pack_blocked_kernel, gpack, 256, 0, st, a->Z, Zt, P, d, d_pad, blocked);
  mape_detail::launch(pack_blocked_kernel, gpack, 256, 0, st, a->M, Mt, P, d, d_pad, blocked);
  mape_detail::launch(pack_blocked_kernel, gpack, 256, 0, st, a->V, Vt, P, d, d_pad, blocked);
  MAPE_LAUNCH_CHECK();
  p = TcParams{};
  p.B = a->B; p.span = a->span; p.Zt = Zt; p.Mt = Mt; p.Vt = Vt; p.bias = bias;
  p.n = n; p.d = d; p.P = P; p.n_pad = tile_rows(n, d, id); p.d_pad = d_pad; p.span_pad = pad16(n);
  p.t0 = a->t0; p.T = a->T; p.period = a->period;
  p.lambda1 = a->lambda1; p.lambda2 = a->lambda2; p.lr = a->lr; p.eps = a->eps;
  p.beta1 = (float)a->beta1; p.beta2 = (float)a->beta2;
  p.omb1 = (float)(1.0 - a->beta1); p.omb2 = (float)(1.0 - a->beta2);
  p.cand = a->cand; p.ldc = a->ldc; p.cap = a->cand_cap; p.count = a->cand_count; p.flags = a->flags;
  p.dbg_phi = a->dbg_phi; p.dbg_grad = a->dbg_grad;
  p.nterms = nterms;
  p.use_bb = tc_use_bb(p.n_pad, p.d_pad, p.nterms, p.span_pad);
  // at least 116 KB of shared memory keeps one CTA per SM, so the 512-column
  // TMEM allocation never waits for another CTA
  smem = smem_layout(p.n_pad, p.d_pad, p.nterms, p.use_bb, p.span_pad).total;
  if (smem < 116 * 1024) smem = 116 * 1024;
  return MAPE_OK;
}

static int tc_unpack(const TcParams& p, const mape_extract_args* a, cudaStream_t st) {
  const unsigned gun = (unsigned)ceil_div((int64_t)a->P * a->d, 256);
  mape_detail::launch(unpack_blocked_kernel, gun, 256, 0, st, p.Zt, a->Z, a->P, a->d, p.d_pad);
  mape_detail::launch(unpack_blocked_kernel, gun, 256, 0, st, p.Mt, a->M, a->P, a->d, p.d_pad);
  mape_detail::launch(unpack_blocked_kernel, gun, 256, 0, st, p.Vt, a->V, a->P, a->d, p.d_pad);
  MAPE_LAUNCH_CHECK();
  return MAPE_OK;
}

// the FP32 state fits in the free TMEM lanes when its three d_pad-wide blocks
// fit in 512 columns
static bool tc_resident_state(const TcParams& p) { return 3 * p.d_pad <= kTmemCols; }

int extract_tc(const mape_extract_args* a, cudaStream_t st) {
  const int d = a->d;
  if (a->T > (1 << 20)) return MAPE_ERR_SHAPE;
  // which kernel: identity-topped B or general B (the flag word is the
  // workspace's last piece)
  Carver cv(a->workspace, a->workspace_bytes);
  const int64_t blocked = ceil_div(a->P, kTileM) * kTileM * (int64_t)pad16(d);
  for (int k = 0; k < 3; ++k) cv.take<float>((size_t)blocked);
  cv.take<float2>((size_t)1 << 20);
  int32_t* idflag = cv.take<int32_t>(1);
  if (!cv.ok) return MAPE_ERR_CAPACITY;
  MAPE_CUDA_TRY(cudaMemsetAsync(idflag, 0, sizeof(int32_t), st));
  mape_detail::launch(identity_top_kernel, (unsigned)ceil_div((int64_t)d * d, 256), 256, 0, st, a->B, d, idflag);
  MAPE_LAUNCH_CHECK();
  int32_t h_notid = 1;
  MAPE_CUDA_TRY(cudaMemcpyAsync(&h_notid, idflag, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  const bool id = h_notid == 0;
  TcParams p;
  uint32_t smem = 0;
  int rc = tc_prepare(a, id, st, p, smem);
  if (rc != MAPE_OK) return rc;
  const bool res = tc_resident_state(p);
  auto kern = id ? (res ? extract_tc_kernel<true, true> : extract_tc_kernel<true, false>)
                 : (res ? extract_tc_kernel<false, true> : extract_tc_kernel<false, false>);
  {
    size_t lim = 0;
    const int rc = allow_max_dynamic_smem((const void*)kern, &lim);
    if (rc != MAPE_OK) return rc;
    if ((size_t)smem > lim) return MAPE_ERR_SHAPE;
  }
  mape_detail::timed_launch(MAPE_TIMED_RESIDENT, st,
                            [&] { mape_detail::launch(kern, (unsigned)ceil_div(a->P, kTileM), kThreads, smem, st, p); });
  MAPE_LAUNCH_CHECK();
  return tc_unpack(p, a, st);
}

struct TcBatch {
  struct Launch {
    int variant = 0;  // bit 0: identity-topped B, bit 1: state in TMEM
    int64_t first = 0, ctas = 0;
    uint32_t smem = 0;
  };
  std::vector<Launch> launches;
  void* table = nullptr;
  void* work = nullptr;
  std::vector<const mape_extract_args*> items;
  std::vector<TcParams> params;
};

static void (*batch_kernel(int v))(const TcParams*, const int2*) {
  switch (v) {
    case 0: return extract_tc_batch_kernel<false, false>;
    case 1: return extract_tc_batch_kernel<true, false>;
    case 2: return extract_tc_batch_kernel<false, true>;
    default: return extract_tc_batch_kernel<true, true>;
  }
}

void extract_tc_batch_free(TcBatch* b) { delete b; }

bool extract_tc_fits(const mape_extract_args* a, bool id) {
  return tc_fits(a->n, a->d, a->precision == MAPE_PREC_BF16X1 ? 1 : 2, id);
}

size_t extract_tc_batch_workspace(const mape_extract_args* const* items, int count) {
  Sizer s;
  int64_t tiles = 0;
  for (int i = 0; i < count; ++i) tiles += ceil_div(items[i]->P, kTileM);
  s.take<TcParams>((size_t)count);
  s.take<int2>((size_t)tiles);
  return s.bytes();
}

// Every call of `items` (resident-kernel shapes; ids[i]: B identity-topped) in
// as few launches as kernel variants: one persistent launch per variant over
// all the variant's tiles.  prepare (uploads; synchronises `st` once) and
// enqueue (launches only: capturable into a CUDA graph).
int extract_tc_batch_prepare(const mape_extract_args* const* items, const bool* ids, int count, void* ws,
                             size_t ws_bytes, cudaStream_t st, TcBatch** out) {
  *out = nullptr;
  std::unique_ptr<TcBatch> hold(new TcBatch());
  TcBatch& plan = *hold;
  std::vector<TcParams> params((size_t)count);
  std::vector<uint32_t> smem((size_t)count);
  for (int i = 0; i < count; ++i) {
    int rc = tc_prepare(items[i], ids[i], st, params[i], smem[i]);
    if (rc != MAPE_OK) return rc;
  }
  Carver cv(ws, ws_bytes);
  TcParams* dtab = cv.take<TcParams>((size_t)count);
  int64_t tiles = 0;
  for (int i = 0; i < count; ++i) tiles += ceil_div(items[i]->P, kTileM);
  int2* dwork = cv.take<int2>((size_t)tiles);
  if (!cv.ok) return MAPE_ERR_CAPACITY;
  // work lists grouped by variant: (identity-topped, state in TMEM)
  std::vector<int2> work;
  work.reserve((size_t)tiles);
  for (int v = 0; v < 4; ++v) {
    const bool vid = v & 1, vres = (v >> 1) & 1;
    TcBatch::Launch L{};
    L.variant = v;
    L.first = (int64_t)work.size();
    for (int i = 0; i < count; ++i) {
      if (ids[i] != vid || tc_resident_state(params[i]) != vres) continue;
      for (int t = 0; t < ceil_div(items[i]->P, kTileM); ++t) work.push_back(make_int2(i, t));
      L.smem = std::max(L.smem, smem[i]);
    }
    L.ctas = (int64_t)work.size() - L.first;
    if (L.ctas > 0) plan.launches.push_back(L);
  }
  MAPE_CUDA_TRY(cudaMemcpyAsync(dtab, params.data(), sizeof(TcParams) * count, cudaMemcpyHostToDevice, st));
  MAPE_CUDA_TRY(cudaMemcpyAsync(dwork, work.data(), sizeof(int2) * work.size(), cudaMemcpyHostToDevice, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  plan.table = dtab;
  plan.work = dwork;
  plan.items.assign(items, items + count);
  plan.params = std::move(params);
  for (auto& L : plan.launches) {
    auto kern = batch_kernel(L.variant);
    size_t lim = 0;
    const int rc = allow_max_dynamic_smem((const void*)kern, &lim);
    if (rc != MAPE_OK) return rc;
    if ((size_t)L.smem > lim) return MAPE_ERR_SHAPE;
  }
  *out = hold.release();
  return MAPE_OK;
}

int extract_tc_batch_enqueue(const TcBatch* pl, cudaStream_t st) {
  const TcBatch& plan = *pl;
  for (const auto& L : plan.launches) {
    mape_detail::launch(batch_kernel(L.variant), (unsigned)L.ctas, kThreads, L.smem, st,
                        static_cast<const TcParams*>(plan.table), static_cast<const int2*>(plan.work) + L.first);
    MAPE_LAUNCH_CHECK();
  }
  for (size_t i = 0; i < plan.items.size(); ++i) {
    int rc = tc_unpack(plan.params[i], plan.items[i], st);
    if (rc != MAPE_OK) return rc;
  }
  return MAPE_OK;
}

}  // namespace mape_detail
