// Algorithm 2 (§3.2) on the tensor cores for shapes whose per-tile state and
// basis do not fit on chip (rows of the MMA tile or d above 256, e.g. n = 2000,
// d = 1600): the "streamed" path.  The fused kernel keeps B and a tile's
// z, m, v on chip for all T steps; here every step streams them.
//
// Per step, three kernels over tiles of 128 starts (M = 128 MMAs, FP32
// accumulators in TMEM), with Bm the rows of B that go through the tensor
// cores (the m rows of B' below an identity top, else all n rows):
//   forward  (grid: tile x 256-row block of Bm)  D1 = hi(Z) Bm^T + lo(Z) Bm^T,
//            K = d streamed in chunks of 64 coordinates: z is read from the
//            blocked FP32 state and split into BF16 operands in shared memory,
//            the Bm chunk arrives by a bulk (TMA) copy; S = sign(D1) is written
//            as the BF16 A operand of the gradient.  On collection steps the
//            same pass forms D2 = round(Z) Bm^T (exact: |round z| <= 256, integer
//            partial sums below 2^24) and stages the candidate rows.
//   collect  (one warp per start) the C4, nonzero and changed tests, a slot in
//            the candidate buffer, the row in canonical sign.
//   gradient (grid: tile x 256-coordinate block)  G = S Bm, K = rows of Bm in
//            chunks of 64, both operands by bulk copy into a two-stage ring
//            (one producer thread, one MMA thread); the epilogue adds the
//            identity rows, lambda1 (ceil z + floor z - 2 z) and the inverse-norm
//            term and runs Adam on the FP32 master z, m, v (read and written
//            once per step), forming the per-start reductions of the next step
//            (||z||_inf and its first index, rounding changed, bound test and
//            first nonzero entry of the identity rows) with atomics.
// Operand chunks use the no-swizzle K-major layout of tc_ptx.cuh.  Every
// mbarrier wait is bounded (2 s); on time-out the CTA sets flag 16, skips its
// outputs, drains what it issued and frees its TMEM.
#include "common.cuh"
#include "extract_internal.cuh"
#include "tc_ptx.cuh"

#include <algorithm>
#include <cmath>
#include <memory>
#include <vector>

namespace {
using namespace mape_tc;

constexpr int kTM = 128;       // starts per tile: the MMA M
constexpr int kThreads = 256;  // 8 warps: two per TMEM lane quarter
constexpr int kThreadsF = kThreads + 32;  // forward kernel: plus the issuing warp
constexpr int kKC = 64;        // K chunk
constexpr int kNB = 256;       // the widest N block: the largest MMA N
constexpr int kChunkA = kTM * kKC * 2;        // one 128 x 64 BF16 operand chunk (16 KB)
// shared memory of the two-stage rings for N blocks of width w
__host__ __device__ constexpr int fwd_stage(int w) { return 3 * kChunkA + w * kKC * 2; }  // hi, lo, round(z), Bm chunk
constexpr int kChunkZ = kTM * kKC * 4;  // one 128 x 64 FP32 chunk of the blocked state (32 KB, contiguous)
// forward pass: two operand stages, then two FP32 z stages
__host__ __device__ constexpr int fwd_smem(int w) { return 2 * fwd_stage(w) + 2 * kChunkZ; }
__host__ __device__ constexpr int grad_stage(int w) { return kChunkA + w * kKC * 2; }    // S chunk, Bm chunk
__host__ __device__ constexpr int tmem_cols(int c) { return c <= 32 ? 32 : c <= 64 ? 64 : c <= 128 ? 128 : c <= 256 ? 256 : 512; }
constexpr int kNoNz = 0x7fffffff;
constexpr uint32_t kChanged = 1, kUnexact = 2;

struct StParams {
  int n, d, P, R;       // R: rows of Bm
  int r0;               // row of B held in row 0 of Bm (d for an identity top, else 0)
  int d64, R64;         // padded to the K chunk
  int tiles, nbF, nbG;  // tiles of 128 starts; N blocks over R64 and d64
  int wF, wG;           // N block widths (multiples of 64, at most 256)
  int ldc, mapoff, lds; // candidate pitch; offset of the Bm rows in a staged row; staged pitch
  const uint8_t* BmF;   // forward B operand: [nbF][d64/64][N x 64] chunks (N = Bm rows)
  const uint8_t* BmF8;  // the same in e4m3 (8-bit chunks, MAPE_PREC_FP8)
  int f8;               // 1: the forward product in e4m3 (z scaled per start), D2 stays BF16
  const uint8_t* BmG;   // gradient B operand: [nbG][R64/64][N x 64] chunks (N = coordinates)
  const int32_t* span;
  float* Zt;
  float* Mt;
  float* Vt;            // blocked [tiles][d64/4][128][4]
  uint8_t* S;           // [tiles][R64/64] chunks of sign(Bm z), 128 x 64 BF16
  int8_t* stage;        // [tiles*128][lds] staged candidate rows
  unsigned long long* zkey;  // [2][tiles*128]: (|z|_inf bits << 32) | (~first argmax)
  uint32_t* acc;        // rounding changed / unexact since the last collection
  uint32_t* oob;        // Bm rows of the staged candidate out of the box (C4)
  uint32_t* idw;        // [2][..] identity rows of round(z) out of the box
  int32_t* first;       // [2][..] first nonzero entry of round(z) on the identity rows
  int32_t* first_map;   // general B: first nonzero entry of B round(z)
  const float2* bias;   // (lr / (1 - beta1^t), 1 / sqrt(1 - beta2^t)) per step
  float lambda1, lambda2, eps, beta1, beta2, omb1, omb2;
  int nterms;
  int8_t* cand;
  int64_t cap;
  unsigned long long* count;
  int32_t* flags;
  float* dbg_phi;
  float* dbg_grad;
  int tile0;              // first tile of this launch (the tile range of a launch may be part of the call's)
  const int32_t* sp_rp;   // sparse forward: CSR of Bm, row starts [R + 1]
  const uint16_t* sp_ci;  //   column indices (coordinates)
  const float* sp_rv;     //   values
};

__device__ __forceinline__ int ptot(const StParams& p) { return p.tiles * kTM; }

// ---------------------------------------------------------------- forward

// Barrier among the converter warps of the forward kernel (named barrier 1),
// returning whether any of them passed true
__device__ __forceinline__ bool conv_barrier_or(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(kThreads)
      : "memory");
  return r != 0;
}

// The e4m3 scale of start pg at step s: the power of two 2^(8 - e) with
// ||z||_inf < 2^e (from the step's ||z||_inf word), so that the scaled z lies
// within [-256, 256]; 1 for z = 0.  A power of two is exact, and the sign of
// B (sc z) is that of B z.
__device__ __forceinline__ float f8_scale(const StParams& p, int s, int64_t pg) {
  const unsigned long long k = p.zkey[(int64_t)(s & 1) * ptot(p) + pg];
  const float zinf = __uint_as_float((uint32_t)(k >> 32));
  if (!(zinf > 0.f)) return 1.f;
  int e;
  frexpf(zinf, &e);
  e = max(-100, min(100, 8 - e));
  return ldexpf(1.f, e);
}

// blk: tile * nbF + row block of this CTA.  Warps 0-7 (the converters) turn
// the z chunks into BF16 operands and afterwards read the accumulators; warp 8
// only issues: the Bm chunk copies and the MMAs.  A stage's operands are
// handed over through the ready barrier (one arrival per converter warp), so
// the conversion of chunk c + 1 runs while the MMAs of chunk c are issued.
template <bool kId>
// merged (FP8 forward steps without collection, at most two row blocks):
// one CTA per tile multiplies every row block of Bm (N0 = wF rows into TMEM
// columns [0, wF), the rest after them), so that z is read and converted
// once per tile instead of once per row block.
__device__ __forceinline__ void stream_fwd_body(const StParams& p, const int blk, int s, int fwd, int collect,
                                                int merged = 0) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t bars[8];  // full[2] (Bm copy), done[2] (MMAs), zfull[2] (z copy), ready[2]
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool conv = tid < kThreads;
  const int nbl = merged ? 1 : p.nbF;  // CTAs per tile in this launch
  const int tile = p.tile0 + blk / nbl, rb = merged ? 0 : blk % nbl;
  const int N = merged ? p.R64 : (rb < p.nbF - 1 ? p.wF : p.R64 - p.wF * (p.nbF - 1));
  const int N0 = merged ? p.wF : N, N1 = N - N0;  // merged: the two row blocks' widths
  const int row0 = rb * p.wF;
  const int fstage = fwd_stage(p.wF);
  const uint32_t fcols = (uint32_t)tmem_cols(2 * p.wF);  // D1 at 0, D2 at wF
  const int nk = p.d64 / kKC;
  const int P2 = ptot(p);
  const uint32_t full0 = smem_u32(&bars[0]), done0 = smem_u32(&bars[2]), zfull0 = smem_u32(&bars[4]),
                 ready0 = smem_u32(&bars[6]);

  // buffers of the next step's per-start reductions start empty
  if (rb == 0 && tid < kTM) {
    const int pg = tile * kTM + tid;
    const int nb = ((s + 1) & 1) * P2 + pg;
    p.zkey[nb] = 0ull;
    p.idw[nb] = 0u;
    p.first[nb] = kNoNz;
  }
  if (tid == 0) {
    mbar_init(full0, 1); mbar_init(full0 + 8, 1);
    mbar_init(done0, 1); mbar_init(done0 + 8, 1);
    mbar_init(zfull0, 1); mbar_init(zfull0 + 8, 1);
    mbar_init(ready0, kThreads / 32); mbar_init(ready0 + 8, kThreads / 32);
    s_abort = (*(volatile int32_t*)p.flags & 16) ? 1 : 0;  // an earlier CTA timed out: the call is abandoned
  }
  if (warp == 0) tmem_alloc(smem_u32(&s_tmem), fcols);
  mbar_init_fence();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t idesc = idesc_bf16(kTM, N);
  const uint32_t idesc8 = idesc_e4m3(kTM, N);
  bool ok = s_abort == 0;
  int issued_copies = 0, issued_commits = 0;  // issuer thread
  int issued_z = 0;                           // converter thread 0

  // item i of this thread: 8 coordinates (core matrix kc) of start r, so that
  // a warp writes 512 contiguous bytes of each operand
  const float4* zbase = reinterpret_cast<const float4*>(p.Zt) + (size_t)tile * (p.d64 / 4) * kTM;
  auto item_r = [&](int i) { const int e = tid + kThreads * i; return (e & 7) | ((e >> 6) << 3); };
  auto item_kc = [&](int i) { return ((tid + kThreads * i) >> 3) & 7; };
  // z chunk c (coordinates 64c .. 64c+63 of the tile's 128 starts: 32 KB,
  // contiguous in the blocked layout) goes to z stage c & 1 by bulk copy,
  // one chunk ahead of its conversion
  uint8_t* const zst = smem + 2 * fstage;
  auto copy_z = [&](int c) {
    const int zs = c & 1;
    mbar_arrive_expect_tx(zfull0 + 8 * zs, (uint32_t)kChunkZ);
    bulk_g2s(smem_u32(zst + zs * kChunkZ), zbase + (size_t)c * (kKC / 4) * kTM, (uint32_t)kChunkZ, zfull0 + 8 * zs);
    ++issued_z;
  };
  // the Bm chunk of chunk c goes to stage c & 1, issued one chunk ahead:
  // chunk c + 1 right after chunk c's MMAs, once those of chunk c - 1 have
  // left its stage
  auto copy_bm = [&](int c) {
    const int stg = c & 1;
    uint8_t* Bc = smem + stg * fstage + 3 * kChunkA;
    if (merged) {  // both row blocks' e4m3 chunks, one after the other from the lo slot on
      mbar_arrive_expect_tx(full0 + 8 * stg, (uint32_t)N * kKC);
      bulk_g2s(smem_u32(Bc - 2 * kChunkA), p.BmF8 + (size_t)c * N0 * kKC, (uint32_t)N0 * kKC, full0 + 8 * stg);
      bulk_g2s(smem_u32(Bc - 2 * kChunkA + N0 * kKC), p.BmF8 + (size_t)p.wF * p.d64 + (size_t)c * N1 * kKC,
               (uint32_t)N1 * kKC, full0 + 8 * stg);
    } else if (p.f8) {  // e4m3 chunk (N x 64 bytes) in the stage's unused lo slot; BF16 chunk only for D2
      const bool b16 = collect != 0, b8 = fwd != 0;
      mbar_arrive_expect_tx(full0 + 8 * stg, (uint32_t)N * kKC * ((b16 ? 2 : 0) + (b8 ? 1 : 0)));
      if (b8)
        bulk_g2s(smem_u32(Bc - 2 * kChunkA), p.BmF8 + (size_t)rb * p.wF * p.d64 + (size_t)c * N * kKC,
                 (uint32_t)N * kKC, full0 + 8 * stg);
      if (b16)
        bulk_g2s(smem_u32(Bc), p.BmF + ((size_t)rb * p.wF * p.d64 + (size_t)c * N * kKC) * 2,
                 (uint32_t)N * kKC * 2, full0 + 8 * stg);
    } else {
      mbar_arrive_expect_tx(full0 + 8 * stg, (uint32_t)N * kKC * 2);
      bulk_g2s(smem_u32(Bc), p.BmF + ((size_t)rb * p.wF * p.d64 + (size_t)c * N * kKC) * 2, (uint32_t)N * kKC * 2,
               full0 + 8 * stg);
    }
    ++issued_copies;
  };

  if (ok && conv) {  // ---- converters ----
    if (tid == 0) copy_z(0);
    for (int c = 0; c < nk; ++c) {
      const int stg = c & 1;
      uint8_t* Ahi = smem + stg * fstage;
      uint8_t* Alo = Ahi + kChunkA;
      uint8_t* Ard = Alo + kChunkA;
      bool w = true;
      if (c >= 2) w = mbar_wait_bounded(done0 + 8 * stg, ((c - 2) >> 1) & 1);  // chunk c - 2's MMAs left the stage
      // every converter finished chunk c - 1, so the z stage of chunk c + 1 is free
      if (conv_barrier_or(!w || *(volatile int*)&s_abort)) { ok = false; break; }
      if (tid == 0 && c + 1 < nk) copy_z(c + 1);
      // a time-out here is voted at the next barrier (every converter must
      // reach it); this chunk's operands then go unused
      if (!mbar_wait_bounded(zfull0 + 8 * (c & 1), (c >> 1) & 1)) s_abort = 1;
      const float4* zs4 = reinterpret_cast<const float4*>(zst + (c & 1) * kChunkZ);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = item_r(i), kc = item_kc(i);
        const float4 q0 = zs4[(2 * kc) * kTM + r], q1 = zs4[(2 * kc + 1) * kTM + r];
        const float z8[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
        const uint32_t o = chunk_off(r, kc * 8);
        if (fwd && p.f8) {
          // e4m3 of z scaled by the start's power of two (per-start scale:
          // max |z| lands in [128, 256), inside the e4m3 range of 448)
          const float sc = f8_scale(p, s, (int64_t)tile * kTM + r);
          float v8[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) v8[k] = z8[k] * sc;
          *reinterpret_cast<uint2*>(Ahi + chunk_off8(r, kc * 8)) = pack_e4m3x8(v8);
        } else if (fwd) {
          uint32_t wh[4], wl[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            wh[k] = pack_bf16x2(z8[2 * k], z8[2 * k + 1]);
            const float2 hf = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&wh[k]));
            wl[k] = pack_bf16x2(z8[2 * k] - hf.x, z8[2 * k + 1] - hf.y);
          }
          *reinterpret_cast<uint4*>(Ahi + o) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
          if (p.nterms > 1) *reinterpret_cast<uint4*>(Alo + o) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
        }
        if (collect) {
          uint32_t wr[4];
          float rz[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) rz[k] = rintf(z8[k]);
#pragma unroll
          for (int k = 0; k < 4; ++k) wr[k] = pack_bf16x2(rz[2 * k], rz[2 * k + 1]);
          *reinterpret_cast<uint4*>(Ard + o) = make_uint4(wr[0], wr[1], wr[2], wr[3]);
          // identity rows of the candidate: g_j = round z_j
          const int64_t pg = (int64_t)tile * kTM + r;
          const int j0 = c * kKC + kc * 8;
          if (kId && rb == 0 && pg < p.P && j0 < p.d) {
            int8_t* row = p.stage + pg * p.lds;
            if (j0 + 8 <= p.d) {
              uint32_t bb[2] = {0, 0};
#pragma unroll
              for (int k = 0; k < 8; ++k) bb[k >> 2] |= ((uint32_t)((int)rz[k] & 0xff)) << (8 * (k & 3));
              *reinterpret_cast<uint2*>(row + j0) = make_uint2(bb[0], bb[1]);
            } else {
              for (int k = 0; j0 + k < p.d; ++k) row[j0 + k] = (int8_t)(int)rz[k];
            }
          }
        }
      }
      // the stage's operands go to the issuer (async proxy)
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(ready0 + 8 * stg);
    }
  } else if (ok && tid == kThreads) {  // ---- issuer ----
    copy_bm(0);
    for (int c = 0; c < nk; ++c) {
      const int stg = c & 1;
      const uint32_t A0 = smem_u32(smem + stg * fstage);
      const uint32_t Bc = A0 + 3 * kChunkA;
      if (!mbar_wait_bounded(ready0 + 8 * stg, (c >> 1) & 1) || !mbar_wait_bounded(full0 + 8 * stg, (c >> 1) & 1) ||
          *(volatile int*)&s_abort) {
        s_abort = 1;
        break;
      }
      tc_fence_after();
      if (merged) {  // D1 of both row blocks in e4m3
        const uint32_t B8 = A0 + kChunkA;
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          const uint64_t a = make_desc(A0 + kk * 256, kChunkLbo, kChunk8Sbo);
          mma_e4m3(tmem, a, make_desc(B8 + kk * 256, kChunkLbo, kChunk8Sbo), idesc_e4m3(kTM, N0), (c | kk) ? 1u : 0u);
          mma_e4m3(tmem + (uint32_t)N0, a, make_desc(B8 + N0 * kKC + kk * 256, kChunkLbo, kChunk8Sbo),
                   idesc_e4m3(kTM, N1), (c | kk) ? 1u : 0u);
        }
      } else if (p.f8 && fwd) {  // D1 in e4m3: K = 32 per instruction, two per chunk
        const uint32_t B8 = A0 + kChunkA;
#pragma unroll
        for (int kk = 0; kk < 2; ++kk)
          mma_e4m3(tmem, make_desc(A0 + kk * 256, kChunkLbo, kChunk8Sbo), make_desc(B8 + kk * 256, kChunkLbo, kChunk8Sbo),
                   idesc8, (c | kk) ? 1u : 0u);
      }
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t b = make_desc(Bc + kk * 256, kChunkLbo, kChunkSbo);
        const uint32_t a0 = (c | kk) ? 1u : 0u;
        if (fwd && !p.f8) {
          mma_bf16(tmem, make_desc(A0 + kk * 256, kChunkLbo, kChunkSbo), b, idesc, a0);
          if (p.nterms > 1) mma_bf16(tmem, make_desc(A0 + kChunkA + kk * 256, kChunkLbo, kChunkSbo), b, idesc, 1u);
        }
        if (collect) mma_bf16(tmem + p.wF, make_desc(A0 + 2 * kChunkA + kk * 256, kChunkLbo, kChunkSbo), b, idesc, a0);
      }
      mma_commit(done0 + 8 * stg);
      ++issued_commits;
      if (c + 1 < nk) {
        if (c >= 1 && !mbar_wait_bounded(done0 + 8 * ((c - 1) & 1), ((c - 1) >> 1) & 1)) {
          s_abort = 1;
          break;
        }
        copy_bm(c + 1);
      }
    }
  }
  // the last chunk's MMAs, then the accumulators (every thread takes part in the vote)
  {
    bool w = true;
    if (ok && conv) {
      const int cl = nk - 1;
      w = mbar_wait_bounded(done0 + 8 * (cl & 1), (cl >> 1) & 1);
    }
    if (__syncthreads_or(!w || s_abort || !ok)) ok = false;
  }

  if (ok && conv) {
    tc_fence_after();
    const int q = warp & 3, h = warp >> 2;
    const int r = q * 32 + lane;
    const int64_t pg = (int64_t)tile * kTM + r;
    const bool live = pg < p.P;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    float l1 = 0.f;
    bool out = false;
    int firstc = kNoNz;
    // FP8: the accumulator holds B (sc z); its sign is that of B z
    const float inv_sc = (fwd && p.f8) ? 1.f / f8_scale(p, s, pg) : 1.f;
    for (int ch = h; ch < N / 16; ch += 2) {
      uint32_t v[16];
      if (fwd) {
        tmem_ld16(tmem + lane_base + ch * 16, v);
        tc_wait_ld();
        uint32_t w[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float y0 = __uint_as_float(v[2 * k]), y1 = __uint_as_float(v[2 * k + 1]);
          w[k] = pack_bf16x2((float)mape_sign_f(y0), (float)mape_sign_f(y1));
          l1 += (fabsf(y0) + fabsf(y1)) * inv_sc;
        }
        const int kg = row0 + ch * 16;  // column of S: row of Bm
        uint8_t* Sp = p.S + ((size_t)tile * (p.R64 / kKC) + kg / kKC) * kChunkA;
        *reinterpret_cast<uint4*>(Sp + chunk_off(r, kg % kKC)) = make_uint4(w[0], w[1], w[2], w[3]);
        *reinterpret_cast<uint4*>(Sp + chunk_off(r, kg % kKC + 8)) = make_uint4(w[4], w[5], w[6], w[7]);
      }
      if (collect) {
        tmem_ld16(tmem + lane_base + p.wF + ch * 16, v);
        tc_wait_ld();
        const int i0 = row0 + ch * 16;
        uint32_t pk[4] = {0, 0, 0, 0};
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int i = i0 + k;
          const int g = __float2int_rn(__uint_as_float(v[k]));
          if (i < p.R) {
            const int row = p.r0 + i;
            const int sp = p.span[row];
            if (g > sp || -g > sp) out = true;
            if (!kId && g != 0 && (row << 1) < firstc) firstc = (row << 1) | (g < 0 ? 1 : 0);
          }
          pk[k >> 2] |= ((uint32_t)(g & 0xff)) << (8 * (k & 3));
        }
        // padding rows of Bm are zero, so their entries are 0
        if (live) *reinterpret_cast<uint4*>(p.stage + pg * p.lds + p.mapoff + i0) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      }
    }
    if (live) {
      if (out) atomicOr(&p.oob[pg], 1u);
      if (!kId && firstc != kNoNz) atomicMin(&p.first_map[pg], firstc);
      if (fwd && s == 0 && p.dbg_phi) atomicAdd(&p.dbg_phi[pg], l1);
    }
  } else if (tid == 0) {
    atomicOr(p.flags, 16);
  }
  if (!ok) {  // drain what the copying and issuing threads started before the memory goes away
    if (tid == 0)
      for (int c = 0; c < issued_z; ++c) mbar_wait_bounded(zfull0 + 8 * (c & 1), (c >> 1) & 1);
    if (tid == kThreads) {
      for (int c = 0; c < issued_copies; ++c) mbar_wait_bounded(full0 + 8 * (c & 1), (c >> 1) & 1);
      if (issued_commits > 0) {
        const int cl = issued_commits - 1;
        mbar_wait_bounded(done0 + 8 * (cl & 1), (cl >> 1) & 1);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, fcols);
  }
}

// ---------------------------------------------------------------- sparse forward

// The forward pass for an identity-topped B whose rows below the identity
// (Bm) are sparse: y = Bm z over the compressed rows of Bm on the CUDA cores,
// in FP32 from the exact FP32 z (no BF16 splitting), so a step costs about
// nnz(Bm) fused multiply-adds per start instead of a dense R x d product and
// is bound by reading z once.  Persistent CTAs of 512 threads hold the CSR of
// Bm in shared memory (when it fits; else it is read through L1) and walk over
// groups of 8 starts of a tile: the z of the next group is copied (cp.async,
// 16-byte pieces of the blocked state) into the second of two buffers (rows of
// d64 + 4 floats: the 8 starts of one column fall in 8 different banks) while
// the current group is multiplied out.  Lane (r, q) of warp w forms rows
// i = 4 w + q + 64 k of y for start r; sign(y) is staged as the 8-row group of
// the tile in every 128 x 64 chunk of S (1 KB each) and copied out with
// 16-byte stores.  On collection steps the same pass forms Bm round(z)
// exactly in int32 (|round z| <= 256 and |B| <= 256 are guaranteed as on the
// tensor-core path) and writes the staged candidate rows.  Outputs are those
// of the tensor-core forward: S, the staged rows, the out-of-box word, the
// debug Phi terms and the reset of the next step's per-start words.
constexpr int kSpStarts = 8;
constexpr int kSpThreads = 512;
constexpr int kSpRowsPerRound = (kSpThreads / 32) * 4;

__host__ __device__ constexpr int sp_ld(int d64) { return d64 + 4; }
__host__ __device__ constexpr size_t sp_zbuf(int d64) { return (size_t)kSpStarts * sp_ld(d64) * 4; }
__host__ __device__ constexpr size_t sp_csr_bytes(int R, int nnz) {
  return ((size_t)(R + 1) * 4 + (size_t)nnz * 4 + (size_t)nnz * 2 + 15) / 16 * 16;
}
// shared memory: two z buffers, the S staging area, then the CSR (if staged)
__host__ __device__ constexpr size_t sp_smem(int d64, int R64, size_t csr) {
  return 2 * sp_zbuf(d64) + (size_t)(R64 / kKC) * 1024 + csr;
}

__global__ void __launch_bounds__(kSpThreads, 1) stream_fwd_sparse_kernel(StParams p, int s, int fwd, int collect,
                                                                          int nnz, int csr_smem) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ float s_l1[kSpStarts];
  __shared__ int s_out[kSpStarts];
  const int tid = threadIdx.x;
  constexpr int kGroups = kTM / kSpStarts;
  const int ld = sp_ld(p.d64);
  const int ng4 = p.d64 / 4;
  const int nck = p.R64 / kKC;
  float* zbuf0 = reinterpret_cast<float*>(smem);
  uint8_t* ss = smem + 2 * sp_zbuf(p.d64);
  // CSR of Bm: in shared memory when it fits, else read through L1
  const int32_t* rp = p.sp_rp;
  const float* rv = p.sp_rv;
  const uint16_t* ci = p.sp_ci;
  if (csr_smem) {  // values (16-byte aligned), column indices, row starts
    float* s_rv = reinterpret_cast<float*>(ss + (size_t)nck * 1024);
    uint16_t* s_ci = reinterpret_cast<uint16_t*>(s_rv + nnz);
    int32_t* s_rp = reinterpret_cast<int32_t*>(s_ci + nnz);
    for (int e = tid; e <= p.R; e += kSpThreads) s_rp[e] = p.sp_rp[e];
    for (int e = tid; e < nnz; e += kSpThreads) {
      s_rv[e] = p.sp_rv[e];
      s_ci[e] = p.sp_ci[e];
    }
    rp = s_rp;
    rv = s_rv;
    ci = s_ci;
  }
  const int P2 = ptot(p);
  const int groups = p.tiles * kGroups;
  auto issue_z = [&](int grp, int buf) {  // the z of group grp into buffer buf (one commit group per thread)
    if (grp < groups) {
      const int tile = grp / kGroups, g8 = grp % kGroups;
      const float4* zt = reinterpret_cast<const float4*>(p.Zt) + (size_t)tile * ng4 * kTM + g8 * kSpStarts;
      const uint32_t base = smem_u32(zbuf0) + (uint32_t)(buf * sp_zbuf(p.d64));
      for (int e = tid; e < ng4 * kSpStarts; e += kSpThreads) {
        const int g = e / kSpStarts, r = e % kSpStarts;
        cp_async16(base + (uint32_t)((r * ld + 4 * g) * 4), zt + (size_t)g * kTM + r);
      }
    }
    cp_async_commit();
  };
  const int warp = tid >> 5, lane = tid & 31, r = lane & 7, q = lane >> 3;
  int buf = 0;
  issue_z(blockIdx.x, 0);
  for (int grp = blockIdx.x; grp < groups; grp += gridDim.x, buf ^= 1) {
    const int tile = grp / kGroups, g8 = grp % kGroups;
    const int64_t pg0 = (int64_t)tile * kTM + g8 * kSpStarts;
    if (tid < kSpStarts) {  // buffers of the next step's per-start reductions start empty
      const int64_t nb = (int64_t)((s + 1) & 1) * P2 + pg0 + tid;
      p.zkey[nb] = 0ull;
      p.idw[nb] = 0u;
      p.first[nb] = kNoNz;
      s_l1[tid] = 0.f;
      s_out[tid] = 0;
    }
    issue_z(grp + gridDim.x, buf ^ 1);  // the next group's z, while this one is multiplied out
    cp_async_wait<1>();
    __syncthreads();  // this group's z (every thread's copies) and the CSR are in place
    const float* zs = zbuf0 + (size_t)buf * (sp_zbuf(p.d64) / 4);
    const int64_t pg = pg0 + r;
    const bool live = pg < p.P;
    const float* zr = zs + r * ld;
    int8_t* srow = p.stage + pg * p.lds + p.mapoff;
    float l1 = 0.f;
    bool out = false;
    for (int i = warp * 4 + q; i < p.R64; i += kSpRowsPerRound) {
      float acc0 = 0.f, acc1 = 0.f;
      int g2 = 0;
      if (i < p.R) {
        // rows hold multiples of 4 entries (zero padded): 4 column indices
        // and 4 values per pair of vector loads, 4 independent gathers of z
        float acc2 = 0.f, acc3 = 0.f;
        for (int e = rp[i], e1 = rp[i + 1]; e < e1; e += 4) {
          const uint2 c4 = *reinterpret_cast<const uint2*>(ci + e);
          const float4 v4 = *reinterpret_cast<const float4*>(rv + e);
          const float z0 = zr[c4.x & 0xffff], z1 = zr[c4.x >> 16], z2 = zr[c4.y & 0xffff], z3 = zr[c4.y >> 16];
          acc0 = fmaf(v4.x, z0, acc0);
          acc1 = fmaf(v4.y, z1, acc1);
          acc2 = fmaf(v4.z, z2, acc2);
          acc3 = fmaf(v4.w, z3, acc3);
          if (collect)
            g2 += (int)v4.x * (int)rintf(z0) + (int)v4.y * (int)rintf(z1) + (int)v4.z * (int)rintf(z2) +
                  (int)v4.w * (int)rintf(z3);
        }
        acc0 += acc2;
        acc1 += acc3;
      }
      const float acc = acc0 + acc1;
      if (fwd) {
        const uint16_t sb = acc > 0.f ? (uint16_t)0x3F80 : (acc < 0.f ? (uint16_t)0xBF80 : (uint16_t)0);
        *reinterpret_cast<uint16_t*>(ss + (i >> 6) * 1024 + ((i & 63) >> 3) * 128 + r * 16 + (i & 7) * 2) = sb;
        l1 += fabsf(acc);
      }
      if (collect && i < p.R) {
        const int sp = p.span[p.r0 + i];
        if (g2 > sp || -g2 > sp) out = true;
        if (live) srow[i] = (int8_t)(g2 & 0xff);
      }
    }
    if (fwd && s == 0 && p.dbg_phi) atomicAdd(&s_l1[r], l1);
    if (out) s_out[r] = 1;
    if (collect) {  // identity rows of the staged candidates: round(z) itself
      for (int e = tid; e < kSpStarts * p.d; e += kSpThreads) {
        const int rr = e / p.d, j = e % p.d;
        if (pg0 + rr < p.P) p.stage[(pg0 + rr) * p.lds + j] = (int8_t)((int)rintf(zs[rr * ld + j]) & 0xff);
      }
    }
    __syncthreads();  // S staged; this z buffer is free for the group after next
    if (fwd) {
      for (int e = tid; e < nck * 64; e += kSpThreads) {
        const int c = e >> 6, k = e & 63;
        const uint4 v = reinterpret_cast<const uint4*>(ss + c * 1024)[k];
        reinterpret_cast<uint4*>(p.S + ((size_t)tile * nck + c) * kChunkA + g8 * 1024)[k] = v;
      }
    }
    if (tid < kSpStarts && pg0 + tid < p.P) {
      if (collect && s_out[tid]) atomicOr(&p.oob[pg0 + tid], 1u);
      if (fwd && s == 0 && p.dbg_phi) atomicAdd(&p.dbg_phi[pg0 + tid], s_l1[tid]);
    }
    __syncthreads();  // the S staging area and the per-start words are free for the next group
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------- collect

// blk: block of 8 starts (one warp each)
template <bool kId>
__device__ __forceinline__ void stream_collect_body(const StParams& p, const int blk, int s) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t pg = (int64_t)p.tile0 * kTM + (int64_t)blk * (blockDim.x >> 5) + warp;
  if (pg >= p.P) return;
  const int P2 = ptot(p);
  long long slot = -1;
  int neg = 0;
  if (lane == 0) {
    const uint32_t a = p.acc[pg], o = p.oob[pg];
    const uint32_t idout = kId ? p.idw[(s & 1) * P2 + pg] : 0u;
    const int fz = kId ? p.first[(s & 1) * P2 + pg] : p.first_map[pg];
    if ((a & kChanged) && !o && !idout && fz != kNoNz) {
      if (a & kUnexact) {
        atomicOr(p.flags, 2);
      } else {
        const unsigned long long at = atomicAdd(p.count, 1ull);
        if ((int64_t)at < p.cap) slot = (long long)at;
        else atomicOr(p.flags, 1);
      }
    }
    neg = (fz != kNoNz && (fz & 1)) ? 1 : 0;
    p.acc[pg] = 0u;
    p.oob[pg] = 0u;
    if (!kId) p.first_map[pg] = kNoNz;
  }
  slot = __shfl_sync(0xffffffffu, slot, 0);
  neg = __shfl_sync(0xffffffffu, neg, 0);
  if (slot < 0) return;
  const int8_t* src = p.stage + pg * p.lds;
  int8_t* dst = p.cand + slot * p.ldc;
  for (int b = lane; b < p.ldc; b += 32) {
    int v = 0;
    if (b < p.n) v = (kId && b >= p.d) ? src[p.mapoff + (b - p.d)] : src[b];
    dst[b] = (int8_t)(neg ? -v : v);
  }
}

// ---------------------------------------------------------------- gradient + Adam

// blk: tile * nbG + coordinate block of this CTA
template <bool kId>
__device__ __forceinline__ void stream_grad_body(const StParams& p, const int blk, int s) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t bars[5];  // full[2], done[2], accumulator ready
  __shared__ int32_t s_span[kNB];             // C4 bounds of this block's coordinates
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = p.tile0 + blk / p.nbG, db = blk % p.nbG;
  const int N = db < p.nbG - 1 ? p.wG : p.d64 - p.wG * (p.nbG - 1);
  const int col0 = db * p.wG;
  const int gstage = grad_stage(p.wG);
  const uint32_t gcols = (uint32_t)tmem_cols(p.wG);
  const int nk = p.R64 / kKC;
  const int P2 = ptot(p);
  const uint32_t full0 = smem_u32(&bars[0]), done0 = smem_u32(&bars[2]), accr = smem_u32(&bars[4]);
  if (*(volatile int32_t*)p.flags & 16) return;  // an earlier CTA timed out: the call is abandoned

  if (tid == 0) {
    mbar_init(full0, 1); mbar_init(full0 + 8, 1);
    mbar_init(done0, 1); mbar_init(done0 + 8, 1);
    mbar_init(accr, 1);
    s_abort = 0;
  }
  if (warp == 0) tmem_alloc(smem_u32(&s_tmem), gcols);
  mbar_init_fence();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  int copies = 0, commits = 0;  // issued by the producer / MMA thread

  if (warp == 0 && lane == 0) {  // producer: both operands of chunk c by bulk copy
    for (int c = 0; c < nk; ++c) {
      const int stg = c & 1;
      if (c >= 2 && !mbar_wait_bounded(done0 + 8 * stg, ((c - 2) >> 1) & 1)) {
        s_abort = 1;
        break;
      }
      if (*(volatile int*)&s_abort) break;
      uint8_t* A = smem + stg * gstage;
      uint8_t* Bc = A + kChunkA;
      mbar_arrive_expect_tx(full0 + 8 * stg, (uint32_t)(kChunkA + N * kKC * 2));
      bulk_g2s(smem_u32(A), p.S + ((size_t)tile * nk + c) * kChunkA, kChunkA, full0 + 8 * stg);
      bulk_g2s(smem_u32(Bc), p.BmG + ((size_t)db * p.wG * p.R64 + (size_t)c * N * kKC) * 2, (uint32_t)N * kKC * 2,
               full0 + 8 * stg);
      ++copies;
    }
  } else if (warp == 1 && lane == 0) {  // MMA issuer
    const uint32_t idesc = idesc_bf16(kTM, N);
    int c = 0;
    for (; c < nk; ++c) {
      const int stg = c & 1;
      if (*(volatile int*)&s_abort || !mbar_wait_bounded(full0 + 8 * stg, (c >> 1) & 1)) {
        s_abort = 1;
        break;
      }
      tc_fence_after();
      const uint32_t A = smem_u32(smem + stg * gstage), Bc = A + kChunkA;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        mma_bf16(tmem, make_desc(A + kk * 256, kChunkLbo, kChunkSbo), make_desc(Bc + kk * 256, kChunkLbo, kChunkSbo),
                 idesc, (c | kk) ? 1u : 0u);
      mma_commit(done0 + 8 * stg);
      ++commits;
    }
    if (c == nk) mma_commit(accr);
  }
  __syncwarp();

  // epilogue geometry: warp w reads TMEM lane quarter w % 4 (its 32 starts);
  // the two warps of a quarter take alternate 8-coordinate chunks
  const int q = warp & 3, h = warp >> 2;
  const int r = q * 32 + lane;
  const int64_t pg = (int64_t)tile * kTM + r;
  const bool row_live = pg < p.P;
  const uint32_t lane_base = (uint32_t)(q * 32) << 16;
  const int nch = N / 8;
  float4* const zt = reinterpret_cast<float4*>(p.Zt) + (size_t)tile * (p.d64 / 4) * kTM + r;
  float4* const mt = reinterpret_cast<float4*>(p.Mt) + (size_t)tile * (p.d64 / 4) * kTM + r;
  float4* const vt = reinterpret_cast<float4*>(p.Vt) + (size_t)tile * (p.d64 / 4) * kTM + r;
  auto load_state = [&](int ch, float4(&z)[2], float4(&m)[2], float4(&v)[2]) {
    const size_t g = (size_t)((col0 + ch * 8) / 4) * kTM;
    z[0] = zt[g]; z[1] = zt[g + kTM];
    m[0] = mt[g]; m[1] = mt[g + kTM];
    v[0] = vt[g]; v[1] = vt[g + kTM];
  };
  // the first chunk's state is in flight while the MMAs run
  float4 cz[2], cm[2], cv[2];
  if (h < nch) load_state(h, cz, cm, cv);
  if (kId)
    for (int k = tid; k < N; k += kThreads) s_span[k] = col0 + k < p.d ? p.span[col0 + k] : 0;
  const bool w = mbar_wait_bounded(accr, 0);
  const bool ok = !__syncthreads_or(!w || s_abort);

  if (ok) {
    tc_fence_after();
    const unsigned long long zk = p.zkey[(s & 1) * P2 + pg];
    const float zinf = __uint_as_float((uint32_t)(zk >> 32));
    const int kmax = zk ? (int)(0xffffffffu - (uint32_t)zk) : -1;
    float inv_term = 0.f;
    if (zinf < 1.f && zinf > 0.f) inv_term = -p.lambda2 / (zinf * zinf);  // times sign(z_kmax)
    const float2 ad = p.bias[s];
    const float step = ad.x, rsb2 = ad.y;
    const bool dbg = s == 0 && (p.dbg_phi || p.dbg_grad);
    float nzinf = 0.f, frac = 0.f, l1_id = 0.f;
    int nkmax = kNoNz, first_id = kNoNz;
    bool changed = false, unexact = false, out_id = false;
    for (int ch = h; ch < nch; ch += 2) {
      const int j0 = col0 + ch * 8;
      float4 nz[2] = {cz[0], cz[1]}, nm[2] = {cm[0], cm[1]}, nv[2] = {cv[0], cv[1]};
      if (ch + 2 < nch) load_state(ch + 2, nz, nm, nv);
      uint32_t gv[8];
      tmem_ld8(tmem + lane_base + ch * 8, gv);
      float zc[8] = {cz[0].x, cz[0].y, cz[0].z, cz[0].w, cz[1].x, cz[1].y, cz[1].z, cz[1].w};
      float mc[8] = {cm[0].x, cm[0].y, cm[0].z, cm[0].w, cm[1].x, cm[1].y, cm[1].z, cm[1].w};
      float vc[8] = {cv[0].x, cv[0].y, cv[0].z, cv[0].w, cv[1].x, cv[1].y, cv[1].z, cv[1].w};
      tc_wait_ld();
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int j = j0 + k;
        const bool live = row_live && j < p.d;
        const float z = zc[k];
        const float fl = floorf(z);
        // ceil z + floor z = 2 floor z + [z not an integer]
        float grad = __uint_as_float(gv[k]) + p.lambda1 * (2.f * fl + (z != fl ? 1.f : 0.f) - 2.f * z);
        if (j == kmax) grad += inv_term * (float)mape_sign_f(z);
        if (kId) grad += (float)mape_sign_f(z);  // identity row j of B: sign((Bz)_j) = sign(z_j)
        if (dbg && live) {
          frac += (z - fl) * (ceilf(z) - z);
          if (kId) l1_id += fabsf(z);
          if (p.dbg_grad) p.dbg_grad[pg * p.d + j] = grad;
        }
        const float m = p.beta1 * mc[k] + p.omb1 * grad;
        const float vv = p.beta2 * vc[k] + p.omb2 * grad * grad;
        const float den = (vv > 0.f ? vv * rsqrtf(vv) : 0.f) * rsb2 + p.eps;
        const float znew = z - step * __fdividef(m, den);  // padding coordinates stay at 0
        zc[k] = znew;
        mc[k] = m;
        vc[k] = vv;
        if (live) {
          const float rn = rintf(znew);
          changed |= rn != rintf(z);
          unexact |= fabsf(rn) > 256.f;
          const float a = fabsf(znew);
          if (nkmax == kNoNz || a > nzinf) { nzinf = a; nkmax = j; }
          if (kId) {
            out_id |= fabsf(rn) > (float)s_span[ch * 8 + k];
            if (first_id == kNoNz && rn != 0.f) first_id = (j << 1) | (rn < 0.f ? 1 : 0);
          }
        }
      }
      const size_t g = (size_t)(j0 / 4) * kTM;
      zt[g] = make_float4(zc[0], zc[1], zc[2], zc[3]);
      zt[g + kTM] = make_float4(zc[4], zc[5], zc[6], zc[7]);
      mt[g] = make_float4(mc[0], mc[1], mc[2], mc[3]);
      mt[g + kTM] = make_float4(mc[4], mc[5], mc[6], mc[7]);
      vt[g] = make_float4(vc[0], vc[1], vc[2], vc[3]);
      vt[g + kTM] = make_float4(vc[4], vc[5], vc[6], vc[7]);
      cz[0] = nz[0]; cz[1] = nz[1];
      cm[0] = nm[0]; cm[1] = nm[1];
      cv[0] = nv[0]; cv[1] = nv[1];
    }
    if (row_live) {
      const int nb = ((s + 1) & 1) * P2 + (int)pg;
      if (nkmax != kNoNz)
        atomicMax(&p.zkey[nb], ((unsigned long long)__float_as_uint(nzinf) << 32) | (0xffffffffu - (uint32_t)nkmax));
      const uint32_t fb = (changed ? kChanged : 0u) | (unexact ? kUnexact : 0u);
      if (fb) atomicOr(&p.acc[pg], fb);
      if (kId) {
        if (out_id) atomicOr(&p.idw[nb], 1u);
        if (first_id != kNoNz) atomicMin(&p.first[nb], first_id);
      }
      if (dbg && p.dbg_phi) {
        float add = p.lambda1 * frac + l1_id;
        if (db == 0 && h == 0) add += p.lambda2 * (zinf > 0.f ? fmaxf(1.f / zinf - 1.f, 0.f) : INFINITY);
        atomicAdd(&p.dbg_phi[pg], add);
      }
    }
  } else if (tid == 0) {
    atomicOr(p.flags, 16);
  }
  if (!ok) {  // drain what the producer and the MMA thread issued
    if (warp == 0 && lane == 0)
      for (int c = 0; c < copies; ++c) mbar_wait_bounded(full0 + 8 * (c & 1), (c >> 1) & 1);
    if (warp == 1 && lane == 0 && commits > 0) {
      const int cl = commits - 1;
      mbar_wait_bounded(done0 + 8 * (cl & 1), (cl >> 1) & 1);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, gcols);
  }
}

// ---------------------------------------------------------------- launch wrappers

template <bool kId>
__global__ void __launch_bounds__(kThreadsF, 1) stream_fwd_kernel(StParams p, int s, int fwd, int collect,
                                                                   int merged) {
  stream_fwd_body<kId>(p, blockIdx.x, s, fwd, collect, merged);
}
template <bool kId>
__global__ void stream_collect_kernel(StParams p, int s) {
  stream_collect_body<kId>(p, blockIdx.x, s);
}
template <bool kId>
__global__ void __launch_bounds__(kThreads, 1) stream_grad_kernel(StParams p, int s) {
  stream_grad_body<kId>(p, blockIdx.x, s);
}

// Many instances per launch: CTA b works on block work[b].y of instance
// work[b].x, whose parameters are table[work[b].x] (a CTA that finds an
// instance with fewer steps than the launch's step does nothing).
__device__ __forceinline__ const StParams& load_params(const StParams* table, int item, StParams& s_p) {
  if (threadIdx.x == 0) s_p = table[item];
  __syncthreads();
  return s_p;
}
template <bool kId>
__global__ void __launch_bounds__(kThreadsF, 1) stream_fwd_batch_kernel(const StParams* __restrict__ table,
                                                                       const int2* __restrict__ work, int s, int fwd,
                                                                       int collect) {
  __shared__ StParams s_p;
  const int2 w = work[blockIdx.x];
  stream_fwd_body<kId>(load_params(table, w.x, s_p), w.y, s, fwd, collect);
}
template <bool kId>
__global__ void stream_collect_batch_kernel(const StParams* __restrict__ table, const int2* __restrict__ work, int s) {
  __shared__ StParams s_p;
  const int2 w = work[blockIdx.x];
  stream_collect_body<kId>(load_params(table, w.x, s_p), w.y, s);
}
template <bool kId>
__global__ void __launch_bounds__(kThreads, 1) stream_grad_batch_kernel(const StParams* __restrict__ table,
                                                                        const int2* __restrict__ work, int s) {
  __shared__ StParams s_p;
  const int2 w = work[blockIdx.x];
  stream_grad_body<kId>(load_params(table, w.x, s_p), w.y, s);
}

// ---------------------------------------------------------------- set-up kernels

// Bm in both operand layouts; flags |= 8 (and *bad = 1) if an entry is not
// exact in BF16 (|B_ij| > 256)
__global__ void pack_bm_kernel(const int32_t* __restrict__ B, int d, int R, int r0, int d64, int R64, int nbF,
                               int nbG, int wF, int wG, uint8_t* __restrict__ BmF, uint8_t* __restrict__ BmG,
                               uint8_t* __restrict__ BmF8, int f8, int32_t* bad, int32_t* flags) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)R64 * d64) return;
  const int i = (int)(e / d64), j = (int)(e % d64);
  const int v = (i < R && j < d) ? B[(int64_t)(r0 + i) * d + j] : 0;
  bool inexact = v > 256 || v < -256;
  if (f8) {  // the e4m3 copy of the forward operand; its entries must be exact too
    const __nv_fp8_storage_t q = __nv_cvt_float_to_fp8((float)v, __NV_SATFINITE, __NV_E4M3);
    const __half_raw hr = __nv_cvt_fp8_to_halfraw(q, __NV_E4M3);
    if (__half2float(*reinterpret_cast<const __half*>(&hr)) != (float)v) inexact = true;
    const int rb = i / wF, rl = i % wF;
    const int Nr = rb < nbF - 1 ? wF : R64 - wF * (nbF - 1);
    BmF8[(size_t)rb * wF * d64 + (size_t)(j / kKC) * Nr * kKC + chunk_off8(rl, j % kKC)] = (uint8_t)q;
  }
  if (inexact) {
    atomicOr(bad, 1);
    atomicOr(flags, 8);
  }
  const __nv_bfloat16 hb = __float2bfloat16_rn((float)v);
  const uint16_t hv = *reinterpret_cast<const uint16_t*>(&hb);
  {
    const int rb = i / wF, rl = i % wF;
    const int Nr = rb < nbF - 1 ? wF : R64 - wF * (nbF - 1);
    const size_t off = ((size_t)rb * wF * d64 + (size_t)(j / kKC) * Nr * kKC) * 2 + chunk_off(rl, j % kKC);
    *reinterpret_cast<uint16_t*>(BmF + off) = hv;
  }
  {
    const int gb = j / wG, jl = j % wG;
    const int Nd = gb < nbG - 1 ? wG : d64 - wG * (nbG - 1);
    const size_t off = ((size_t)gb * wG * R64 + (size_t)(i / kKC) * Nd * kKC) * 2 + chunk_off(jl, i % kKC);
    *reinterpret_cast<uint16_t*>(BmG + off) = hv;
  }
}

// [P x d] row-major  <->  blocked [tiles][d64/4][128][4] (zero padded)
// [P x d] row-major <-> blocked [tiles][d64/4][128][4] (zero padded).  Grid
// (tiles, d64 / 8) x 128 threads: thread r moves coordinates 8 y .. 8 y + 7 of
// start x * 128 + r, 32 contiguous bytes of its row (16-byte vector accesses
// when d % 4 == 0 and the row-major array is 16-byte aligned), and the blocked
// side is two float4 rows of 128 starts, coalesced over the threads.
__global__ void pack128_kernel(const float* __restrict__ in, float* __restrict__ out, int P, int d, int d64) {
  const int r = threadIdx.x, g8 = blockIdx.y;
  const int64_t tile = blockIdx.x, row = tile * kTM + r;
  const int j0 = 8 * g8;
  const bool vec = (d & 3) == 0 && ((uintptr_t)in & 15) == 0;
  float v[8];
  if (row < P && j0 + 8 <= d && vec) {
    const float4* src = reinterpret_cast<const float4*>(in + row * d + j0);
    const float4 a = src[0], b = src[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = (row < P && j0 + k < d) ? in[row * d + j0 + k] : 0.f;
  }
  float4* dst = reinterpret_cast<float4*>(out) + (tile * (d64 / 4) + 2 * g8) * kTM + r;
  dst[0] = make_float4(v[0], v[1], v[2], v[3]);
  dst[kTM] = make_float4(v[4], v[5], v[6], v[7]);
}

__global__ void unpack128_kernel(const float* __restrict__ in, float* __restrict__ out, int P, int d, int d64) {
  const int r = threadIdx.x, g8 = blockIdx.y;
  const int64_t tile = blockIdx.x, row = tile * kTM + r;
  const bool vec = (d & 3) == 0 && ((uintptr_t)out & 15) == 0;
  if (row >= P) return;
  const int j0 = 8 * g8;
  const float4* src = reinterpret_cast<const float4*>(in) + (tile * (d64 / 4) + 2 * g8) * kTM + r;
  const float4 a = src[0], b = src[kTM];
  const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
  if (j0 + 8 <= d && vec) {
    float4* dst = reinterpret_cast<float4*>(out + row * d + j0);
    dst[0] = a;
    dst[1] = b;
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (j0 + k < d) out[row * d + j0 + k] = v[k];
  }
}

// per-start words of the first step: ||z0||_inf and its first index, the
// collection state
__global__ void stream_init_kernel(StParams p) {
  const int64_t pg = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int P2 = ptot(p);
  if (pg >= P2) return;
  unsigned long long key = 0ull;
  if (pg < p.P) {
    const int tile = (int)(pg / kTM), r = (int)(pg % kTM);
    const float4* zt = reinterpret_cast<const float4*>(p.Zt) + (size_t)tile * (p.d64 / 4) * kTM + r;
    float best = 0.f;
    int kb = -1;
    for (int g = 0; g < p.d64 / 4; ++g) {
      const float4 q = zt[(size_t)g * kTM];
      const float a4[4] = {fabsf(q.x), fabsf(q.y), fabsf(q.z), fabsf(q.w)};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int j = 4 * g + k;
        if (j < p.d && (kb < 0 || a4[k] > best)) { best = a4[k]; kb = j; }
      }
    }
    key = ((unsigned long long)__float_as_uint(best) << 32) | (0xffffffffu - (uint32_t)kb);
  }
  p.zkey[pg] = key;
  p.zkey[P2 + pg] = 0ull;
  p.acc[pg] = kChanged;  // the first collection of a call always counts
  p.oob[pg] = 0u;
  p.idw[pg] = 0u;
  p.idw[P2 + pg] = 0u;
  p.first[pg] = kNoNz;
  p.first[P2 + pg] = kNoNz;
  p.first_map[pg] = kNoNz;
}

__global__ void stream_identity_top_kernel(const int32_t* __restrict__ B, int d, int32_t* __restrict__ flag) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)d * d) return;
  const int i = (int)(e / d), j = (int)(e % d);
  if (B[(int64_t)i * d + j] != (i == j ? 1 : 0)) atomicOr(flag, 1);
}

// compressed rows of Bm (rows r0 .. r0 + R - 1 of B): nonzeros per row (one
// warp per row) rounded up to a multiple of 4, their exclusive prefix (one
// block), the entries in column order followed by zero entries
__global__ void bm_count_kernel(const int32_t* __restrict__ B, int d, int R, int r0, int32_t* __restrict__ cnt) {
  const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (i >= R) return;
  int c = 0;
  for (int j = lane; j < d; j += 32) c += B[(int64_t)(r0 + i) * d + j] != 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) cnt[i] = (c + 3) & ~3;  // rows padded to 4 entries: vector loads of the sparse forward
}

__global__ void bm_scan_kernel(const int32_t* __restrict__ cnt, int R, int32_t* __restrict__ rp) {
  __shared__ int32_t s_part[1024];
  const int t = threadIdx.x, per = (R + 1023) / 1024;
  const int a = t * per, b = min(a + per, R);
  int32_t sum = 0;
  for (int i = a; i < b; ++i) sum += cnt[i];
  s_part[t] = sum;
  __syncthreads();
  if (t == 0) {
    int32_t run = 0;
    for (int k = 0; k < 1024; ++k) {
      const int32_t v = s_part[k];
      s_part[k] = run;
      run += v;
    }
  }
  __syncthreads();
  int32_t run = s_part[t];
  for (int i = a; i < b; ++i) {
    rp[i] = run;
    run += cnt[i];
  }
  if (b == R && a < b) rp[R] = run;
  if (R == 0 && t == 0) rp[0] = 0;
}

__global__ void bm_fill_kernel(const int32_t* __restrict__ B, int d, int R, int r0, const int32_t* __restrict__ rp,
                               uint16_t* __restrict__ ci, float* __restrict__ rv) {
  const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (i >= R) return;
  int pos = rp[i];
  for (int j0 = 0; j0 < d; j0 += 32) {
    const int j = j0 + lane;
    const int v = j < d ? B[(int64_t)(r0 + i) * d + j] : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, v != 0);
    if (v != 0) {
      const int at = pos + __popc(bal & ((1u << lane) - 1));
      ci[at] = (uint16_t)j;
      rv[at] = (float)v;
    }
    pos += __popc(bal);
  }
  for (int e = pos + lane; e < rp[i + 1]; e += 32) {  // the row's padding: column 0, value 0
    ci[e] = 0;
    rv[e] = 0.f;
  }
}

int r64(int x) { return (x + kKC - 1) / kKC * kKC; }
int r16(int x) { return (x + 15) / 16 * 16; }

struct StreamShape {
  int R, r0, d64, R64, tiles, nbF, nbG, wF, wG, mapoff, lds;
};

StreamShape stream_shape(int n, int d, int P, bool id, int wF = kNB, int wG = kNB) {
  StreamShape s{};
  s.R = id ? n - d : n;
  s.r0 = id ? d : 0;
  s.d64 = r64(d);
  s.R64 = s.R > 0 ? r64(s.R) : kKC;
  s.tiles = (int)mape_detail::ceil_div(P, kTM);
  s.wF = wF;
  s.wG = wG;
  s.nbF = (int)mape_detail::ceil_div(s.R64, wF);
  s.nbG = (int)mape_detail::ceil_div(s.d64, wG);
  s.mapoff = id ? r16(d) : 0;
  s.lds = s.mapoff + s.R64;
  return s;
}

// elementwise maximum of the layouts of a general and an identity-topped B:
// the workspace is sized before B is inspected
StreamShape stream_bound(int n, int d, int P) {
  StreamShape g = stream_shape(n, d, P, false), i = stream_shape(n, d, P, true);
  g.R64 = g.R64 > i.R64 ? g.R64 : i.R64;
  g.lds = g.lds > i.lds ? g.lds : i.lds;
  return g;
}

constexpr int32_t kBiasSteps = 1 << 20;  // bias-correction table: up to 2^20 steps per call
constexpr int kSplitTiles = 64;          // calls of at least this many tiles run as two halves on two streams

// The sparse forward is used while nnz(Bm) <= R d / 16 (density at most 1/16).
constexpr int kSparseDensityInv = 16;
size_t sp_capacity(const StreamShape& sh) { return (size_t)sh.R64 * sh.d64 / kSparseDensityInv + 4 * (size_t)sh.R64 + 1; }

template <typename Carve>
void carve_stream(Carve& cv, const StreamShape& sh) {
  const size_t P2 = (size_t)sh.tiles * kTM;
  const size_t blocked = P2 * sh.d64;
  for (int k = 0; k < 3; ++k) cv.template take<float>(blocked);
  cv.template take<uint8_t>(P2 * sh.R64 * 2);             // S
  cv.template take<int8_t>(P2 * sh.lds);                  // staged rows
  cv.template take<uint8_t>((size_t)sh.R64 * sh.d64 * 2); // BmF
  cv.template take<uint8_t>((size_t)sh.R64 * sh.d64 * 2); // BmG
  cv.template take<uint8_t>((size_t)sh.R64 * sh.d64);     // BmF8
  cv.template take<unsigned long long>(2 * P2);           // zkey
  cv.template take<uint32_t>(P2);                         // acc
  cv.template take<uint32_t>(P2);                         // oob
  cv.template take<uint32_t>(2 * P2);                     // idw
  cv.template take<int32_t>(2 * P2);                      // first
  cv.template take<int32_t>(P2);                          // first_map
  cv.template take<float2>((size_t)kBiasSteps);           // bias table
  cv.template take<int32_t>(2);                           // identity flag, inexact flag
  cv.template take<int32_t>((size_t)sh.R64 + 1);          // sparse forward: nonzeros per row of Bm
  cv.template take<int32_t>((size_t)sh.R64 + 1);          //   row starts
  cv.template take<uint16_t>(sp_capacity(sh));            //   column indices
  cv.template take<float>(sp_capacity(sh));               //   values
}

}  // namespace

namespace mape_detail {

bool extract_stream_supported(int32_t n, int32_t d) { return n <= 4096 && d <= 4096; }

// sized for a general B (all n rows through the tensor cores), which covers
// the identity-topped case
size_t extract_stream_workspace(int32_t n, int32_t d, int32_t P) {
  if (!extract_stream_supported(n, d)) return 0;
  Sizer s;
  carve_stream(s, stream_bound(n, d, P));
  return s.bytes();
}

// One call's pieces of its workspace, carved with the bounding layout.
struct StCarved {
  StreamShape sh;
  float *Zt, *Mt, *Vt;
  uint8_t *S, *BmF, *BmG, *BmF8;
  int8_t* stage;
  unsigned long long* zkey;
  uint32_t *acc, *oob, *idw;
  int32_t *first, *first_map, *hflags;
  float2* bias;
  int32_t *sp_cnt, *sp_rp;
  uint16_t* sp_ci;
  float* sp_rv;
};

static int st_carve(const mape_extract_args* a, bool id, StCarved& c) {
  const int n = a->n, d = a->d, P = a->P;
  if (a->T > kBiasSteps || !extract_stream_supported(n, d)) return MAPE_ERR_SHAPE;
  const StreamShape gen = stream_bound(n, d, P);
  Carver cv(a->workspace, a->workspace_bytes);
  const size_t P2 = (size_t)gen.tiles * kTM;
  c.Zt = cv.take<float>(P2 * gen.d64);
  c.Mt = cv.take<float>(P2 * gen.d64);
  c.Vt = cv.take<float>(P2 * gen.d64);
  c.S = cv.take<uint8_t>(P2 * gen.R64 * 2);
  c.stage = cv.take<int8_t>(P2 * gen.lds);
  c.BmF = cv.take<uint8_t>((size_t)gen.R64 * gen.d64 * 2);
  c.BmG = cv.take<uint8_t>((size_t)gen.R64 * gen.d64 * 2);
  c.BmF8 = cv.take<uint8_t>((size_t)gen.R64 * gen.d64);
  c.zkey = cv.take<unsigned long long>(2 * P2);
  c.acc = cv.take<uint32_t>(P2);
  c.oob = cv.take<uint32_t>(P2);
  c.idw = cv.take<uint32_t>(2 * P2);
  c.first = cv.take<int32_t>(2 * P2);
  c.first_map = cv.take<int32_t>(P2);
  c.bias = cv.take<float2>((size_t)kBiasSteps);
  c.hflags = cv.take<int32_t>(2);
  c.sp_cnt = cv.take<int32_t>((size_t)gen.R64 + 1);
  c.sp_rp = cv.take<int32_t>((size_t)gen.R64 + 1);
  c.sp_ci = cv.take<uint16_t>(sp_capacity(gen));
  c.sp_rv = cv.take<float>(sp_capacity(gen));
  if (!cv.ok) return MAPE_ERR_CAPACITY;
  c.sh = stream_shape(n, d, P, id);
  return MAPE_OK;
}

// B in both operand layouts; hflags[1] = 1 (and flags |= 8) if B is not exact in BF16
static int st_pack_b(const StCarved& c, const mape_extract_args* a, cudaStream_t st) {
  const StreamShape& sh = c.sh;
  MAPE_CUDA_TRY(cudaMemsetAsync(c.hflags + 1, 0, sizeof(int32_t), st));
  const int f8 = (a->precision & MAPE_PREC_MASK) == MAPE_PREC_FP8 ? 1 : 0;
  launch(pack_bm_kernel, (unsigned)ceil_div((int64_t)sh.R64 * sh.d64, 256), 256, 0, st, a->B, a->d, sh.R, sh.r0,
         sh.d64, sh.R64, sh.nbF, sh.nbG, sh.wF, sh.wG, c.BmF, c.BmG, c.BmF8, f8, c.hflags + 1, a->flags);
  MAPE_LAUNCH_CHECK();
  return MAPE_OK;
}

// bias table, blocked state, staged rows, per-start words; the parameters
static int st_setup(const StCarved& c, const mape_extract_args* a, cudaStream_t st, StParams& p) {
  const StreamShape& sh = c.sh;
  const int n = a->n, d = a->d, P = a->P;
  std::vector<float2> bc((size_t)a->T);
  for (int s = 0; s < a->T; ++s) {
    const double t = (double)a->t0 + s + 1;
    const double bc1 = 1.0 - std::pow(a->beta1, t), bc2 = 1.0 - std::pow(a->beta2, t);
    bc[s] = make_float2((float)((double)a->lr / bc1), (float)(1.0 / std::sqrt(bc2)));
  }
  MAPE_CUDA_TRY(cudaMemcpyAsync(c.bias, bc.data(), sizeof(float2) * bc.size(), cudaMemcpyHostToDevice, st));
  const size_t P2 = (size_t)sh.tiles * kTM;
  const dim3 gpack((unsigned)sh.tiles, (unsigned)(sh.d64 / 8));
  launch(pack128_kernel, gpack, kTM, 0, st, a->Z, c.Zt, P, d, sh.d64);
  launch(pack128_kernel, gpack, kTM, 0, st, a->M, c.Mt, P, d, sh.d64);
  launch(pack128_kernel, gpack, kTM, 0, st, a->V, c.Vt, P, d, sh.d64);
  MAPE_CUDA_TRY(cudaMemsetAsync(c.stage, 0, P2 * sh.lds, st));
  if (a->dbg_phi) MAPE_CUDA_TRY(cudaMemsetAsync(a->dbg_phi, 0, sizeof(float) * P, st));
  p = StParams{};
  p.n = n; p.d = d; p.P = P; p.R = sh.R; p.r0 = sh.r0; p.d64 = sh.d64; p.R64 = sh.R64;
  p.tiles = sh.tiles; p.nbF = sh.nbF; p.nbG = sh.nbG; p.wF = sh.wF; p.wG = sh.wG;
  p.ldc = a->ldc; p.mapoff = sh.mapoff; p.lds = sh.lds;
  p.BmF = c.BmF; p.BmG = c.BmG; p.span = a->span; p.Zt = c.Zt; p.Mt = c.Mt; p.Vt = c.Vt; p.S = c.S;
  p.stage = c.stage; p.zkey = c.zkey; p.acc = c.acc; p.oob = c.oob; p.idw = c.idw; p.first = c.first;
  p.first_map = c.first_map; p.bias = c.bias;
  p.lambda1 = a->lambda1; p.lambda2 = a->lambda2; p.eps = a->eps;
  p.beta1 = (float)a->beta1; p.beta2 = (float)a->beta2;
  p.omb1 = (float)(1.0 - a->beta1); p.omb2 = (float)(1.0 - a->beta2);
  p.nterms = (a->precision & MAPE_PREC_MASK) == MAPE_PREC_BF16 ? 2 : 1;
  p.f8 = (a->precision & MAPE_PREC_MASK) == MAPE_PREC_FP8 ? 1 : 0;
  p.BmF8 = c.BmF8;
  p.cand = a->cand; p.cap = a->cand_cap; p.count = a->cand_count; p.flags = a->flags;
  p.dbg_phi = a->dbg_phi; p.dbg_grad = a->dbg_grad;
  launch(stream_init_kernel, (unsigned)ceil_div((int64_t)P2, 256), 256, 0, st, p);
  MAPE_LAUNCH_CHECK();
  return MAPE_OK;
}

static int st_unpack(const StCarved& c, const mape_extract_args* a, cudaStream_t st) {
  const dim3 gun((unsigned)c.sh.tiles, (unsigned)(c.sh.d64 / 8));
  launch(unpack128_kernel, gun, kTM, 0, st, c.Zt, a->Z, a->P, a->d, c.sh.d64);
  launch(unpack128_kernel, gun, kTM, 0, st, c.Mt, a->M, a->P, a->d, c.sh.d64);
  launch(unpack128_kernel, gun, kTM, 0, st, c.Vt, a->V, a->P, a->d, c.sh.d64);
  MAPE_LAUNCH_CHECK();
  return MAPE_OK;
}

// The forward pass's shared memory (at least 115 KB: three operand chunks
// and a B chunk per stage) keeps it at one CTA per SM, so its TMEM (2 wF
// columns, at most 512) always fits; the gradient pass holds wG columns per
// CTA and its registers (about 116 per thread) keep it at two CTAs per SM.
static int st_attributes(bool batch) {
  for (int id = 0; id < 2; ++id) {
    const void* f = batch ? (id ? (const void*)stream_fwd_batch_kernel<true> : (const void*)stream_fwd_batch_kernel<false>)
                          : (id ? (const void*)stream_fwd_kernel<true> : (const void*)stream_fwd_kernel<false>);
    const void* g = batch ? (id ? (const void*)stream_grad_batch_kernel<true> : (const void*)stream_grad_batch_kernel<false>)
                          : (id ? (const void*)stream_grad_kernel<true> : (const void*)stream_grad_kernel<false>);
    MAPE_CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, fwd_smem(kNB)));
    MAPE_CUDA_TRY(cudaFuncSetAttribute(g, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * grad_stage(kNB)));
  }
  return MAPE_OK;
}

// the steps a call of T steps from t0 takes: forward (+ collection of the
// previous rounding when due), gradient; the last rounding when due
template <typename Fwd, typename Coll, typename Grad>
static void st_schedule(int t0, int T, int period, Fwd fwd, Coll coll, Grad grad) {
  for (int s = 0; s < T; ++s) {
    const int t = t0 + s + 1;
    const int collect = (s >= 1 && (t - 1) % period == 0) ? 1 : 0;
    fwd(s, 1, collect);
    if (collect) coll(s);
    grad(s);
  }
  if ((t0 + T) % period == 0) {
    fwd(T, 0, 1);
    coll(T);
  }
}

int extract_stream_widths(const mape_extract_args* a, cudaStream_t st, int wF, int wG, int fwd_mode) {
  const int d = a->d, P = a->P;
  if (wF < kKC || wF > kNB || wF % kKC || wG < kKC || wG > kNB || wG % kKC) return MAPE_ERR_INVALID_ARG;
  StCarved c;
  int rc = st_carve(a, false, c);
  if (rc != MAPE_OK) return rc;
  MAPE_CUDA_TRY(cudaMemsetAsync(c.hflags, 0, sizeof(int32_t), st));
  launch(stream_identity_top_kernel, (unsigned)ceil_div((int64_t)d * d, 256), 256, 0, st, a->B, d, c.hflags);
  MAPE_LAUNCH_CHECK();
  int32_t h_notid = 1;
  MAPE_CUDA_TRY(cudaMemcpyAsync(&h_notid, c.hflags, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  const bool id = h_notid == 0;
  c.sh = stream_shape(a->n, d, P, id, wF, wG);
  if ((rc = st_pack_b(c, a, st)) != MAPE_OK) return rc;
  // the sparse forward: asked for, an identity-topped B, z carried in full
  // (not the one-term BF16 precision), and Bm at density at most 1/16
  if (fwd_mode == kFwdSparse && (!id || (a->precision & MAPE_PREC_MASK) != MAPE_PREC_BF16)) return MAPE_ERR_SHAPE;
  const bool want_sparse = fwd_mode == kFwdSparse;
  if (want_sparse) {
    const unsigned gw = (unsigned)ceil_div((int64_t)c.sh.R * 32, 256);
    launch(bm_count_kernel, gw, 256, 0, st, a->B, d, c.sh.R, c.sh.r0, c.sp_cnt);
    launch(bm_scan_kernel, 1, 1024, 0, st, c.sp_cnt, c.sh.R, c.sp_rp);
    MAPE_LAUNCH_CHECK();
  }
  int32_t h_bad = 0, h_nnz = 0;
  MAPE_CUDA_TRY(cudaMemcpyAsync(&h_bad, c.hflags + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  if (want_sparse) MAPE_CUDA_TRY(cudaMemcpyAsync(&h_nnz, c.sp_rp + c.sh.R, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  if (h_bad) return MAPE_OK;  // flag 8 is set; nothing runs, nothing is collected
  // h_nnz counts the rows' padding to multiples of 4 (at most 3 per row)
  const int64_t nnz_lo = std::max<int64_t>(0, (int64_t)h_nnz - 3 * (int64_t)c.sh.R);
  const bool sparse = want_sparse && (size_t)h_nnz <= sp_capacity(c.sh) &&
                      nnz_lo * kSparseDensityInv <= (int64_t)c.sh.R * d;
  if (want_sparse && !sparse) return MAPE_ERR_SHAPE;
  StParams p;
  if ((rc = st_setup(c, a, st, p)) != MAPE_OK) return rc;
  if ((rc = st_attributes(false)) != MAPE_OK) return rc;
  const StreamShape& sh = c.sh;
  const unsigned gF = (unsigned)(sh.tiles * sh.nbF), gG = (unsigned)(sh.tiles * sh.nbG);
  const unsigned gC = (unsigned)ceil_div(P, 8);
  auto fwdk = id ? stream_fwd_kernel<true> : stream_fwd_kernel<false>;
  auto gradk = id ? stream_grad_kernel<true> : stream_grad_kernel<false>;
  auto collk = id ? stream_collect_kernel<true> : stream_collect_kernel<false>;
  const int fsm = fwd_smem(sh.wF), gsm = 2 * grad_stage(sh.wG);
  // sparse forward: persistent CTAs, one per SM; the CSR joins their shared
  // memory when the total stays within 200 KB
  int dev = 0, nsm = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int groups = sh.tiles * (kTM / kSpStarts);
  const unsigned gS = (unsigned)std::min(groups, nsm);
  const size_t csr = sp_csr_bytes(sh.R, h_nnz);
  const int csr_in_smem = sp_smem(sh.d64, sh.R64, csr) <= (size_t)200 * 1024 ? 1 : 0;
  const size_t ssm = sp_smem(sh.d64, sh.R64, csr_in_smem ? csr : 0);
  if (sparse) {
    if (ssm > (size_t)227 * 1024) return MAPE_ERR_SHAPE;
    const unsigned gw = (unsigned)ceil_div((int64_t)sh.R * 32, 256);
    launch(bm_fill_kernel, gw, 256, 0, st, a->B, d, sh.R, sh.r0, c.sp_rp, c.sp_ci, c.sp_rv);
    size_t lim = 0;
    if ((rc = allow_max_dynamic_smem((const void*)stream_fwd_sparse_kernel, &lim)) != MAPE_OK) return rc;
    if (ssm > lim) return MAPE_ERR_SHAPE;
    p.sp_rp = c.sp_rp;
    p.sp_ci = c.sp_ci;
    p.sp_rv = c.sp_rv;
  }
  if (sparse) {
    st_schedule(
        a->t0, a->T, a->period,
        [&](int s, int f, int col) {
          timed_launch(MAPE_TIMED_STREAM_FWD, st, [&] {
            launch(stream_fwd_sparse_kernel, gS, kSpThreads, ssm, st, p, s, f, col, h_nnz, csr_in_smem);
          });
        },
        [&](int s) { timed_launch(MAPE_TIMED_STREAM_COLLECT, st, [&] { launch(collk, gC, 256, 0, st, p, s); }); },
        [&](int s) { timed_launch(MAPE_TIMED_STREAM_GRAD, st, [&] { launch(gradk, gG, kThreads, gsm, st, p, s); }); });
    MAPE_LAUNCH_CHECK();
    return st_unpack(c, a, st);
  }
  // The tiles are independent problems, so with enough of them the call runs
  // as two halves on two streams (the second joins the caller's stream at the
  // end): the forward pass of one half, bound by moving z through shared
  // memory, runs beside the gradient pass of the other, bound by HBM.
  const int nhalf = sh.tiles >= kSplitTiles ? 2 : 1;
  cudaStream_t st2 = st;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  if (nhalf == 2) {
    MAPE_CUDA_TRY(cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking));
    MAPE_CUDA_TRY(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
    MAPE_CUDA_TRY(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
    MAPE_CUDA_TRY(cudaEventRecord(ev_fork, st));
    MAPE_CUDA_TRY(cudaStreamWaitEvent(st2, ev_fork, 0));
  }
  struct Half {
    StParams p;
    cudaStream_t st;
    unsigned gF, gG, gC;
  };
  Half H[2];
  const int tA = nhalf == 2 ? sh.tiles / 2 : sh.tiles;
  for (int hh = 0; hh < nhalf; ++hh) {
    const int t0 = hh == 0 ? 0 : tA, nt = hh == 0 ? tA : sh.tiles - tA;
    H[hh].p = p;
    H[hh].p.tile0 = t0;
    H[hh].st = hh == 0 ? st : st2;
    H[hh].gF = (unsigned)(nt * sh.nbF);
    H[hh].gG = (unsigned)(nt * sh.nbG);
    const int64_t starts = std::min<int64_t>(P, (int64_t)(t0 + nt) * kTM) - (int64_t)t0 * kTM;
    H[hh].gC = (unsigned)ceil_div(std::max<int64_t>(starts, 1), 8);
  }
  // FP8 steps without collection: one CTA per tile over both row blocks
  const bool can_merge = p.f8 && sh.nbF == 2 && sh.wF == kNB && sh.R64 <= 2 * kNB;
  auto fwd = [&](const Half& h, int s, int f, int col) {
    const int merged = (can_merge && f && !col) ? 1 : 0;
    const unsigned g = merged ? h.gF / (unsigned)sh.nbF : h.gF;
    timed_launch(MAPE_TIMED_STREAM_FWD, h.st, [&] { launch(fwdk, g, kThreadsF, fsm, h.st, h.p, s, f, col, merged); });
  };
  auto coll = [&](const Half& h, int s) {
    timed_launch(MAPE_TIMED_STREAM_COLLECT, h.st, [&] { launch(collk, h.gC, 256, 0, h.st, h.p, s); });
  };
  auto grad = [&](const Half& h, int s) {
    timed_launch(MAPE_TIMED_STREAM_GRAD, h.st, [&] { launch(gradk, h.gG, kThreads, gsm, h.st, h.p, s); });
  };
  // the halves' launches interleaved step by step, in st_schedule's order
  for (int s = 0; s < a->T; ++s) {
    const int t = a->t0 + s + 1;
    const int collect = (s >= 1 && (t - 1) % a->period == 0) ? 1 : 0;
    for (int hh = 0; hh < nhalf; ++hh) {
      fwd(H[hh], s, 1, collect);
      if (collect) coll(H[hh], s);
      grad(H[hh], s);
    }
  }
  if ((a->t0 + a->T) % a->period == 0)
    for (int hh = 0; hh < nhalf; ++hh) {
      fwd(H[hh], a->T, 0, 1);
      coll(H[hh], a->T);
    }
  MAPE_LAUNCH_CHECK();
  if (nhalf == 2) {
    MAPE_CUDA_TRY(cudaEventRecord(ev_join, st2));
    MAPE_CUDA_TRY(cudaStreamWaitEvent(st, ev_join, 0));
    cudaEventDestroy(ev_fork);
    cudaEventDestroy(ev_join);
    cudaStreamDestroy(st2);  // released once its work has completed
  }
  return st_unpack(c, a, st);
}

int extract_stream(const mape_extract_args* a, cudaStream_t st, int fwd_mode) {
  return extract_stream_widths(a, st, kNB, kNB, fwd_mode);
}

struct StBatch {
  struct Class {  // the calls of one basis kind (identity-topped or general)
    bool id = false;
    StParams* table = nullptr;
    int2 *wF = nullptr, *wC = nullptr, *wG = nullptr;
    int64_t nF = 0, nC = 0, nG = 0;
  };
  std::vector<Class> classes;
  std::vector<const mape_extract_args*> items;
  std::vector<StCarved> carved;
  std::vector<bool> run;  // false: B not exact in BF16 (flag 8 set, nothing runs)
  int t0 = 0, T = 0, period = 1;
};

void extract_stream_batch_free(StBatch* b) { delete b; }

int identity_tops(const mape_extract_args* const* items, int count, int32_t* dflags, cudaStream_t st,
                  std::vector<bool>& ids) {
  ids.assign((size_t)count, false);
  if (count == 0) return MAPE_OK;
  MAPE_CUDA_TRY(cudaMemsetAsync(dflags, 0, sizeof(int32_t) * count, st));
  for (int i = 0; i < count; ++i) {
    const int d = items[i]->d;
    launch(stream_identity_top_kernel, (unsigned)ceil_div((int64_t)d * d, 256), 256, 0, st, items[i]->B, d, dflags + i);
  }
  MAPE_LAUNCH_CHECK();
  std::vector<int32_t> h((size_t)count, 1);
  MAPE_CUDA_TRY(cudaMemcpyAsync(h.data(), dflags, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  for (int i = 0; i < count; ++i) ids[i] = h[i] == 0;
  return MAPE_OK;
}

size_t extract_stream_batch_workspace(const mape_extract_args* const* items, int count) {
  Sizer s;
  int64_t nF = 0, nC = 0, nG = 0;
  for (int i = 0; i < count; ++i) {
    const StreamShape b = stream_bound(items[i]->n, items[i]->d, items[i]->P);
    const int64_t nbF = ceil_div(b.R64, kNB);
    nF += (int64_t)b.tiles * nbF;
    nG += (int64_t)b.tiles * b.nbG;
    nC += ceil_div(items[i]->P, 8);
  }
  for (int k = 0; k < 2; ++k) {  // per basis kind
    s.take<StParams>((size_t)count);
    s.take<int2>((size_t)nF);
    s.take<int2>((size_t)nC);
    s.take<int2>((size_t)nG);
  }
  return s.bytes();
}

int extract_stream_batch_prepare(const mape_extract_args* const* items, const bool* ids, int count, void* ws,
                                 size_t ws_bytes, cudaStream_t st, StBatch** out) {
  *out = nullptr;
  std::unique_ptr<StBatch> plan(new StBatch());
  plan->items.assign(items, items + count);
  plan->carved.resize((size_t)count);
  plan->run.assign((size_t)count, true);
  if (count > 0) {
    plan->t0 = items[0]->t0;
    plan->T = items[0]->T;
    plan->period = items[0]->period;
  }
  int rc;
  for (int i = 0; i < count; ++i) {
    if ((rc = st_carve(items[i], ids[i], plan->carved[i])) != MAPE_OK) return rc;
    if ((rc = st_pack_b(plan->carved[i], items[i], st)) != MAPE_OK) return rc;
  }
  std::vector<int32_t> bad((size_t)count, 0);
  for (int i = 0; i < count; ++i)
    MAPE_CUDA_TRY(cudaMemcpyAsync(&bad[i], plan->carved[i].hflags + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  Carver cv(ws, ws_bytes);
  for (int k = 0; k < 2; ++k) {
    const bool id = k == 1;
    std::vector<StParams> table;
    std::vector<int2> wF, wC, wG;
    for (int i = 0; i < count; ++i) {
      if (ids[i] != id) continue;
      if (bad[i]) { plan->run[i] = false; continue; }
      StParams p;
      if ((rc = st_setup(plan->carved[i], items[i], st, p)) != MAPE_OK) return rc;
      const int slot = (int)table.size();
      table.push_back(p);
      for (int b = 0; b < p.tiles * p.nbF; ++b) wF.push_back(make_int2(slot, b));
      for (int b = 0; b < p.tiles * p.nbG; ++b) wG.push_back(make_int2(slot, b));
      for (int b = 0; b < (int)ceil_div(p.P, 8); ++b) wC.push_back(make_int2(slot, b));
    }
    StBatch::Class C;
    C.id = id;
    C.table = cv.take<StParams>((size_t)count);
    C.wF = cv.take<int2>(wF.size());
    C.wC = cv.take<int2>(wC.size());
    C.wG = cv.take<int2>(wG.size());
    if (!cv.ok) return MAPE_ERR_CAPACITY;
    if (table.empty()) continue;
    C.nF = (int64_t)wF.size(); C.nC = (int64_t)wC.size(); C.nG = (int64_t)wG.size();
    MAPE_CUDA_TRY(cudaMemcpyAsync(C.table, table.data(), sizeof(StParams) * table.size(), cudaMemcpyHostToDevice, st));
    MAPE_CUDA_TRY(cudaMemcpyAsync(C.wF, wF.data(), sizeof(int2) * wF.size(), cudaMemcpyHostToDevice, st));
    MAPE_CUDA_TRY(cudaMemcpyAsync(C.wC, wC.data(), sizeof(int2) * wC.size(), cudaMemcpyHostToDevice, st));
    MAPE_CUDA_TRY(cudaMemcpyAsync(C.wG, wG.data(), sizeof(int2) * wG.size(), cudaMemcpyHostToDevice, st));
    plan->classes.push_back(C);
  }
  MAPE_CUDA_TRY(cudaStreamSynchronize(st));
  if ((rc = st_attributes(true)) != MAPE_OK) return rc;
  *out = plan.release();
  return MAPE_OK;
}

int extract_stream_batch_enqueue(const StBatch* plan, cudaStream_t st) {
  for (const auto& C : plan->classes) {
    auto fwdk = C.id ? stream_fwd_batch_kernel<true> : stream_fwd_batch_kernel<false>;
    auto gradk = C.id ? stream_grad_batch_kernel<true> : stream_grad_batch_kernel<false>;
    auto collk = C.id ? stream_collect_batch_kernel<true> : stream_collect_batch_kernel<false>;
    st_schedule(
        plan->t0, plan->T, plan->period,
        [&](int s, int f, int col) {
          launch(fwdk, (unsigned)C.nF, kThreadsF, fwd_smem(kNB), st, C.table, C.wF, s, f, col);
        },
        [&](int s) { launch(collk, (unsigned)C.nC, 256, 0, st, C.table, C.wC, s); },
        [&](int s) { launch(gradk, (unsigned)C.nG, kThreads, 2 * grad_stage(kNB), st, C.table, C.wG, s); });
    MAPE_LAUNCH_CHECK();
  }
  for (size_t i = 0; i < plan->items.size(); ++i) {
    if (!plan->run[i]) continue;
    int rc = st_unpack(plan->carved[i], plan->items[i], st);
    if (rc != MAPE_OK) return rc;
  }
  return MAPE_OK;
}

}  // namespace mape_detail
