// Split-precision pole sum on the tcgen05 tensor cores (far poles) and the
// FP64 near-pole window.
//
// The pole sum of Eq. 1 is the product of Eq. 2 in the packed form
//   R(p, e) = (1/2a) sum_k P_pk D_ke,  P_pk = w_ik w_jk (p = (i <= j)),
//   D_ke = 1 / (E_k - E_e),
// a GEMM with M = pairs, K = poles, N = energies.  Neither operand exists in
// global memory: each CTA forms its tile of P from TMA-staged rows of W and
// its tile of D from the pole and energy values, in shared memory.
//
// Precision: both operands are scaled by powers of two to [-256, 256] (P per
// pair, D per energy), formed in double-float (FP32 hi + lo, about 46 bits),
// and cut into four slices: the nearest integer, the next 8 bits (multiples
// of 2^-8), the next 8 bits (multiples of 2^-16) and the rest rounded to BF16.
// The first three are exact in BF16; the last leaves an error below 2^-34 of
// the scale.  Thirteen slice products are accumulated on the tensor cores:
// all ten with u + v <= 3 and the three order-4 products (1,3), (2,2), (3,1)
// that the four slices provide.  They go to four FP32 TMEM accumulators, one
// per order (order 4 shares the order-3 one); orders 0-2 hold values on a
// fixed grid, so their FP32 sums are exact while below 2^24 of that grid.
// Every 2048 poles the accumulators are drained into double-float running
// sums (FP32 hi + lo) by error-free additions (TwoSum), on the FP32 pipe: the
// sums keep about 48 bits, and the FP64 pipe stays out of the drain.  With
// five slices (15 products, the default) the low parts are kept in the
// order-3 TMEM columns, which the next period's order-3 products add onto,
// and only the high parts in registers.
//
// Two forms of the MMAs: one-SM (tcgen05 cta_group::1; CTA clusters share P or
// D slices through distributed shared memory) and, for 1 x 2 clusters with D
// by TMA and 15 products, 2-SM (cta_group::2 on a CTA pair: M = 256 energies,
// each SM reading its own D slices and the P slices of the 64 pairs it forms).
// Both sum the same products in the same order per accumulator.
//
// Poles with |E_k - E_e| < delta are excluded from the GEMM by per-energy pole
// index ranges [klo, khi) and summed in FP64 by the near-window kernel, so the
// two parts partition the pole set exactly.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <algorithm>
#include <cstring>
#include <vector>
#include <cudaTypedefs.h>

#include "rm_internal.cuh"
#include "tc_ptx.cuh"

namespace rm {

namespace {

constexpr int BM = 128;                 // pairs per tile: 8 i-channels x 16 j-channels
constexpr int BN = 128;                 // energies per tile
constexpr int KS = 32;                  // poles per k-step (64-byte BF16 rows)
constexpr int NWORK = 16;               // producer / drain warps
constexpr int NTHREADS = (NWORK + 3) * 32;  // + MMA issue warp + cluster copy warp + D-slice loader warp
constexpr int DRAIN_KSTEPS = 64;        // drain every 2048 poles
constexpr int SLICE_BYTES = BM * KS * 2;          // 8 KB: 128 rows x 64 B
constexpr int WI_FLOATS = 16 * KS;   // 8 channels x (hi, lo) rows
constexpr int WJ_FLOATS = 32 * KS;   // 16 channels x (hi, lo) rows
constexpr int PO_FLOATS = 2 * KS;    // poles hi row, lo row
constexpr int TX_BYTES = (WI_FLOATS + WJ_FLOATS + PO_FLOATS) * 4;  // 6400
// Shared-memory geometry for NS slices per operand.  Without RING a stage holds NS slices of P
// (A), NS of D (B) and the staged W rows and poles: four slices fit three stages in the 227 KB
// of a CTA, five only two.  With RING (five slices, D by TMA) the D slices live in a ring of
// their own, two deep, and the stages (P slices + W rows) stay three deep: 3 x 47 + 2 x 40 KB.
template <int NS, bool RING = false>
struct TcGeo {
  static constexpr int A_BYTES = NS * SLICE_BYTES;
  static constexpr int B_BYTES = NS * SLICE_BYTES;
  static constexpr int STAGES = (NS == 5 && !RING) ? 2 : 3;
  static constexpr int BSTAGES = RING ? 2 : STAGES;  // D-slice buffers
  static constexpr int W_OFF = RING ? A_BYTES : A_BYTES + B_BYTES;  // W rows within a stage
  static constexpr int STAGE_STRIDE = ((W_OFF + TX_BYTES + 1023) / 1024) * 1024;
  static constexpr int B_RING = RING ? STAGES * STAGE_STRIDE : 0;  // offset of the D ring
  static constexpr int BARS_OFF = STAGES * STAGE_STRIDE + (RING ? BSTAGES * B_BYTES : 0);
  static constexpr int NBARS = 5 * STAGES + 3 + (RING ? BSTAGES : 0);
  static constexpr size_t SMEM = (size_t)BARS_OFF + 1024 + NBARS * 8 + 16;
};
static_assert(TcGeo<4>::SMEM <= 232448 && TcGeo<5>::SMEM <= 232448 && TcGeo<5, true>::SMEM <= 232448,
              "a CTA's shared memory");
// slices per operand of a product set: 3 products use two, 6 three, 10 and 13 four, 15 five
__host__ __device__ constexpr int slices_of(int nprod) { return nprod == 3 ? 2 : (nprod == 6 ? 3 : (nprod == 15 ? 5 : 4)); }
constexpr long long WAIT_BUDGET = 4000000000LL;   // clock cycles (~2 s) per mbarrier wait

static_assert(BM == 128 && BN == 128, "TMEM layout assumes 128 x 128 tiles");

// byte offset of element (row r, k) in a K-major, 64-byte-swizzled slice
__device__ __forceinline__ uint32_t swz(int r, int k) {
  return (uint32_t)((r >> 3) * 512 + (r & 7) * 64 + ((((k >> 3) ^ ((r >> 1) & 3))) << 4) + ((k & 7) << 1));
}

// x = xh + xl (double-float, |x| <= 256) -> four slices: nearest integer,
// then multiples of 2^-8 and of 2^-16, then the rest.  s0..s2 are exact in
// BF16; s3 (|s3| <= 2^-17) is rounded to BF16 when packed.
__device__ __forceinline__ void slice4(float xh, float xl, float (&s)[4]) {
  const float h0 = __fsub_rn(__fadd_rn(xh, 12582912.0f), 12582912.0f);  // nearest integer
  const float h1 = __fsub_rn(__fadd_rn(xh, 49152.0f), 49152.0f);        // nearest multiple of 2^-8
  s[0] = h0;
  s[1] = __fsub_rn(h1, h0);
  const float r = __fadd_rn(__fsub_rn(xh, h1), xl);
  s[2] = __fsub_rn(__fadd_rn(r, 192.0f), 192.0f);                       // nearest multiple of 2^-16
  s[3] = __fsub_rn(r, s[2]);
}

// (ah + al)(bh + bl) -> (ph, pl), double-float product (error ~2^-46 relative)
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& ph, float& pl) {
  ph = __fmul_rn(ah, bh);
  const float e = __fmaf_rn(ah, bh, -ph);
  pl = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, e));
}

// 1 / ((kh + kl) - (eh + el)) as a double-float
__device__ __forceinline__ void df_recip_diff(float kh, float kl, float eh, float el, float& rh, float& rl) {
  // two-difference of the high parts, then add the low parts
  const float s = __fsub_rn(kh, eh);
  const float bb = __fsub_rn(s, kh);
  const float err = __fsub_rn(__fsub_rn(kh, __fsub_rn(s, bb)), __fadd_rn(eh, bb));
  const float dl0 = __fadd_rn(err, __fsub_rn(kl, el));
  const float dh = __fadd_rn(s, dl0);
  const float dl = __fsub_rn(dl0, __fsub_rn(dh, s));
  // approximate reciprocal (1 ulp); the residual correction below absorbs its error
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rh) : "f"(dh));
  float c = __fmaf_rn(-dh, rh, 1.0f);  // exact residual 1 - dh * rh
  c = __fmaf_rn(-dl, rh, c);
  rl = __fmul_rn(rh, c);
}

// s + e = a + b exactly (round to nearest, no overflow): Knuth's TwoSum
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// x = xh + xl (double-float, |x| <= 256) -> five slices: the nearest integer, then multiples of
// 2^-8, 2^-16 and 2^-24, then the rest.  s0..s3 hold at most 8 significant bits each and are
// exact in BF16; s4 (|s4| <= 2^-25) is rounded to BF16 when packed (error 2^-34, 2^-42 of the
// scale).  The remainder after s1 is carried as an exact double-float (TwoSum), so that the
// 2^-24 slice is not limited by the rounding of one FP32 addition.
__device__ __forceinline__ void slice5(float xh, float xl, float (&s)[5]) {
  const float h0 = __fsub_rn(__fadd_rn(xh, 12582912.0f), 12582912.0f);  // nearest integer
  const float h1 = __fsub_rn(__fadd_rn(xh, 49152.0f), 49152.0f);        // nearest multiple of 2^-8
  s[0] = h0;
  s[1] = __fsub_rn(h1, h0);
  float rh, rl;
  two_sum(__fsub_rn(xh, h1), xl, rh, rl);                                // rh + rl = x - h1 exactly
  s[2] = __fsub_rn(__fadd_rn(rh, 192.0f), 192.0f);                       // nearest multiple of 2^-16
  const float r2 = __fadd_rn(__fsub_rn(rh, s[2]), rl);                   // |r2| <= 2^-17
  s[3] = __fsub_rn(__fadd_rn(r2, 0.75f), 0.75f);                         // nearest multiple of 2^-24
  s[4] = __fsub_rn(r2, s[3]);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// The slices s0..s2 sit on grids 1, 2^-8, 2^-16 with at most 8 significant
// bits, so they are exact in FP16 as well (the 2^-16 grid lies in FP16's
// subnormal range, spacing 2^-24); s3 is rounded to 2^-24 there.
__device__ __forceinline__ uint32_t pack_f16x2(float lo, float hi) {
  __half2 v = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t pack_slice(float lo, float hi, bool f16) {
  return f16 ? pack_f16x2(lo, hi) : pack_bf16x2(lo, hi);
}

// The four packed slices of D for the poles (k, k + 1) = (ph0 + pl0, ph1 + pl1) at the energy
// eh + el: 1 / (E_k - E) in double-float, scaled by m0, m1 (0 for a near-window or padding pole),
// cut into slices, word v holding slice v of both poles.  The producers and the D-slice kernel
// both use it, so the two ways of staging D give the same bits.
__device__ __forceinline__ void d_pack(float ph0, float pl0, float ph1, float pl1, float eh, float el, float m0,
                                       float m1, bool f16, uint32_t (&w)[4]) {
  float rh0, rl0, rh1, rl1;
  df_recip_diff(ph0, pl0, eh, el, rh0, rl0);
  df_recip_diff(ph1, pl1, eh, el, rh1, rl1);
  float s0[4], s1[4];
  slice4(__fmul_rn(rh0, m0), __fmul_rn(rl0, m0), s0);
  slice4(__fmul_rn(rh1, m1), __fmul_rn(rl1, m1), s1);
#pragma unroll
  for (int v = 0; v < 4; ++v) w[v] = pack_slice(s0[v], s1[v], f16);
}

// As d_pack with five BF16 slices (the 15-product set).
__device__ __forceinline__ void d_pack5(float ph0, float pl0, float ph1, float pl1, float eh, float el, float m0,
                                        float m1, uint32_t (&w)[5]) {
  float rh0, rl0, rh1, rl1;
  df_recip_diff(ph0, pl0, eh, el, rh0, rl0);
  df_recip_diff(ph1, pl1, eh, el, rh1, rl1);
  float s0[5], s1[5];
  slice5(__fmul_rn(rh0, m0), __fmul_rn(rl0, m0), s0);
  slice5(__fmul_rn(rh1, m1), __fmul_rn(rl1, m1), s1);
#pragma unroll
  for (int v = 0; v < 5; ++v) w[v] = pack_bf16x2(s0[v], s1[v]);
}

// One half h (16 cells) of a drain of the 15-product accumulators: the exact sums of orders 0-2
// go into the high parts Vh[0..15] by TwoSum (error-free), lo = (order-3 column) + the three
// TwoSum errors, in that order, and (Vh, lo) is renormalised by one more TwoSum.  The order-3
// column holds the previous low part plus this period's order-3 and order-4 products (the MMAs
// accumulate onto it), so the low parts never sit in registers across the k-loop.
__device__ __forceinline__ void drain_half(uint32_t trow, int h, float (&Vh)[16], float (&lo)[16]) {
  float t[16];
#pragma unroll
  for (int o = 0; o < 3; ++o) {
    uint32_t r[16];
    ptx::tmem_ld16(trow + (uint32_t)(o * 128 + h * 16), r);
    ptx::tmem_wait_ld();
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      float sh, se;
      two_sum(Vh[c], __uint_as_float(r[c]), sh, se);
      Vh[c] = sh;
      t[c] = o == 0 ? se : __fadd_rn(t[c], se);
    }
  }
  uint32_t r[16];
  ptx::tmem_ld16(trow + (uint32_t)(384 + h * 16), r);
  ptx::tmem_wait_ld();
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    // renormalised (exactly, TwoSum) so that the low part carried into the next period is at
    // most half an ulp of the high part: the order-3 products then accumulate onto the smallest
    // possible value (the tensor cores' FP32 accumulation loses more on a larger one)
    float sh, se;
    two_sum(Vh[c], __fadd_rn(__uint_as_float(r[c]), t[c]), sh, se);
    Vh[c] = sh;
    lo[c] = se;
  }
}

struct TCArgs {
  const float* mult_p;
  const double* f_p;
  const int32_t* klo;
  const int32_t* khi;
  const double* tau;
  const float* mult_e;
  const float* Eh;
  const float* El;
  const int2* tiles;
  int n, N, nK;
  int f16;          // slices in FP16 instead of BF16
  int nprod;        // slice products per far term: 3, 6, 10 or 13
  long long wait_budget;  // clock cycles a single mbarrier wait may take before the tile aborts
  int64_t e_begin;  // absolute index of the chunk's first energy
  int ne;           // energies in the chunk
  double* R;        // [ne * np]
  int32_t* err;
};

// One 128-pair x 128-energy output tile: pairs from i-block I0 (8 channels) and
// j-block J0 (16 channels), energies n0 .. n0+127 of the chunk that starts at
// absolute energy index g.e_begin and holds g.ne energies.
//
// Cluster sharing (CX x CY CTAs, rank = rx + CX ry): the CX CTAs of one
// cluster row hold different pair tiles of one wave and the same energy tile,
// the CY CTAs of one cluster column the same pair tile and different energy
// tiles.  Each CTA forms 1/CX of the D slices (energy rows) and 1/CY of the P
// slices (pair rows) of a k-step in its own stage buffer; once they are
// written (barrier `gen`), a copy warp forwards those contiguous row blocks to
// the same place in the stage buffers of the CTAs that share them, by bulk
// copies into distributed shared memory that complete as transaction bytes on
// the receivers' `full` barriers.  Slice formation per CTA thus shrinks to
// 1/CX + 1/CY of a full tile while the MMAs stay local.  A stage is empty
// when the MMAs of every CTA that it feeds are done (their commits are
// multicast to the senders).
//
// DT: the D slices of the chunk were written to global memory by the D-slice
// kernel (the same arithmetic, d_pack) and come in by TMA, one 3-D box (32
// poles x 128 energies x 4 slices) per k-step, issued by one producer thread
// once the stage is empty and completing on dfull; the producers form only P,
// and clusters share P alone (CX = 1).
//
// NS: slices per operand the tile's shared memory holds (4: the 3-, 6-, 10- and 13-product sets,
// three stages; 5: the 15-product set, two stages, or with D by TMA three stages of P and W rows
// and a two-deep ring of D buffers, refilled by the loading producer thread once the MMAs of the
// step two back are done).
template <int CX, int CY, bool DT, int NS>
__device__ __forceinline__ void tc_tile(const CUtensorMap* map_omega, const CUtensorMap* map_pol,
                                        const CUtensorMap* map_d, const TCArgs& g, int I0, int J0, int n0,
                                        unsigned char* smem_raw) {
  using namespace ptx;
  static_assert(NS == 4 || NS == 5, "four or five slices per operand");
  constexpr bool RING = NS == 5 && DT;  // D slices in a two-deep ring of their own
  using Geo = TcGeo<NS, RING>;
  constexpr int STAGES = Geo::STAGES;
  constexpr int BST = Geo::BSTAGES;
  static_assert(!RING || BST == 2, "the D ring is two deep");
  constexpr int A_BYTES = Geo::A_BYTES;
  constexpr int B_BYTES = Geo::B_BYTES;
  constexpr int W_OFF = Geo::W_OFF;
  constexpr int STAGE_STRIDE = Geo::STAGE_STRIDE;
  constexpr int NBARS = Geo::NBARS;
  constexpr int CL = CX * CY;
  static_assert(!DT || CX == 1, "TMA-staged D slices are not shared across the cluster");
  static_assert(CX == 1 || CX == 2 || CX == 4, "CX in {1, 2, 4}");
  static_assert(CY == 1 || CY == 2 || CY == 4, "CY in {1, 2, 4}");
  static_assert(CX * CY <= 8, "portable cluster size");
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Geo::BARS_OFF);
  uint64_t* full = bars;
  uint64_t* empty = bars + STAGES;
  uint64_t* wfull = bars + 2 * STAGES;
  uint64_t* gen = bars + 3 * STAGES;
  uint64_t* dfull = bars + 4 * STAGES;
  uint64_t* acc_full = bars + 5 * STAGES;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* done = acc_full + 2;
  uint64_t* emptyB = acc_full + 3;  // RING: the MMAs of a step are done with its D buffer
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + NBARS);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nK = g.nK;
  const int n = g.n;

  // cluster position and the CTAs this one exchanges slices with (itself included)
  uint32_t rank = 0;
  if constexpr (CL > 1) rank = cluster_ctarank();
  const int rx = (int)rank % CX, ry = (int)rank / CX;
  uint32_t peer_mask = 0;
#pragma unroll
  for (int q = 0; q < CL; ++q)
    if (q % CX == rx || q / CX == ry) peer_mask |= 1u << q;
  constexpr int NPEERS = CX + CY - 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full + s, CL > 1 ? 1 : NWORK);  // clusters: the copy warp's arrive + incoming bytes
      mbar_init(empty + s, NPEERS);
      mbar_init(wfull + s, 1);
      mbar_init(gen + s, NWORK);
      mbar_init(dfull + s, 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, NWORK);
    mbar_init(done, 1);
    if constexpr (RING)
      for (int q = 0; q < BST; ++q) mbar_init(emptyB + q, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == NWORK) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  if constexpr (CL > 1) cluster_sync();  // peers' barriers are initialised before any remote arrive
  else __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == NWORK) {
    // ------------------------------------------------ TMA + MMA issue (1 thread)
    if (lane == 0) {
      int tma_last[STAGES];
      for (int s = 0; s < STAGES; ++s) tma_last[s] = -1;
      auto issue_tma = [&](int s, int j) {
        uint8_t* st = smem + s * STAGE_STRIDE;
        float* WI = reinterpret_cast<float*>(st + W_OFF);
        float* WJ = WI + WI_FLOATS;
        float* PO = WJ + WJ_FLOATS;
        mbar_arrive_expect_tx(wfull + s, TX_BYTES);
        const int x = j * KS;
        tma_load_2d(WI, map_omega, wfull + s, x, 2 * I0);
        tma_load_2d(WJ, map_omega, wfull + s, x, 2 * J0);
        tma_load_2d(WJ + 16 * KS, map_omega, wfull + s, x, 2 * J0 + 16);
        tma_load_2d(PO, map_pol, wfull + s, x, 0);
        tma_last[s] = j;
      };
      for (int s = 0; s < STAGES && s < nK; ++s) issue_tma(s, s);
      const uint32_t idN256 = idesc_bf16_f32(128, 256, g.f16 != 0);
      const uint32_t idN128 = idesc_bf16_f32(128, 128, g.f16 != 0);
      const int nprod = g.nprod;
      bool ok = true;
      bool issued = false;
      for (int j = 0; j < nK; ++j) {
        const int s = j % STAGES;
        bool got;
        if constexpr (CL > 1) got = mbar_wait_cluster(full + s, (uint32_t)((j / STAGES) & 1), abort_flag, g.wait_budget);
        else got = mbar_wait(full + s, (uint32_t)((j / STAGES) & 1), abort_flag, g.wait_budget);
        if constexpr (RING) {
          if (got) got = mbar_wait(dfull + j % BST, (uint32_t)((j / BST) & 1), abort_flag, g.wait_budget);
        } else {
          if (got && DT) got = mbar_wait(dfull + s, (uint32_t)((j / STAGES) & 1), abort_flag, g.wait_budget);
        }
        if (!got) { ok = false; break; }
        if (j + STAGES < nK) issue_tma(s, j + STAGES);
        const int d = j / DRAIN_KSTEPS;
        const bool first = (j % DRAIN_KSTEPS) == 0;
        if (first && d > 0) {
          if (!mbar_wait(acc_empty, (uint32_t)((d - 1) & 1), abort_flag, g.wait_budget)) { ok = false; break; }
        }
        tc_fence_after();
        const uint32_t a = smem_u32(smem + s * STAGE_STRIDE);
        const uint32_t b = RING ? smem_u32(smem + Geo::B_RING + (j % BST) * B_BYTES) : a + A_BYTES;
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          const uint32_t ko = kk * 32;
          const uint32_t f = (first && kk == 0) ? 0u : 1u;
          auto A = [&](int u) { return desc_kmajor_sw64(a + u * SLICE_BYTES + ko); };
          auto B = [&](int v) { return desc_kmajor_sw64(b + v * SLICE_BYTES + ko); };
          // columns: order 0 [0,128), 1 [128,256), 2 [256,384), 3 [384,512); an N = 256 product
          // q_u x [r_v | r_v+1] writes orders u+v and u+v+1 at once.  The first product into
          // each used accumulator of a drain period starts it (f = 0).
          mma_bf16_ss(tmem + 0, A(0), B(0), idN256, f);  // (0,0) (0,1)
          if constexpr (NS == 5) {
            // all 15 products with u + v <= 4; order 4 shares the order-3 accumulator, which
            // also carries the running sums' low parts from drain to drain, so this product
            // starts orders 2 and 3 only once (the drains zero order 2 instead)
            const uint32_t f23 = (j == 0 && kk == 0) ? 0u : 1u;
            mma_bf16_ss(tmem + 256, A(0), B(2), idN256, f23);  // (0,2) (0,3)
            mma_bf16_ss(tmem + 384, A(0), B(4), idN128, 1u);  // (0,4)
            mma_bf16_ss(tmem + 128, A(1), B(0), idN256, 1u);  // (1,0) (1,1)
            mma_bf16_ss(tmem + 384, A(1), B(2), idN128, 1u);  // (1,2)
            mma_bf16_ss(tmem + 384, A(1), B(3), idN128, 1u);  // (1,3)
            mma_bf16_ss(tmem + 256, A(2), B(0), idN256, 1u);  // (2,0) (2,1)
            mma_bf16_ss(tmem + 384, A(2), B(2), idN128, 1u);  // (2,2)
            mma_bf16_ss(tmem + 384, A(3), B(0), idN128, 1u);  // (3,0)
            mma_bf16_ss(tmem + 384, A(3), B(1), idN128, 1u);  // (3,1)
            mma_bf16_ss(tmem + 384, A(4), B(0), idN128, 1u);  // (4,0)
          } else if (nprod == 3) {
            mma_bf16_ss(tmem + 128, A(1), B(0), idN128, 1u);  // (1,0)
          } else if (nprod == 6) {
            mma_bf16_ss(tmem + 256, A(0), B(2), idN128, f);   // (0,2)
            mma_bf16_ss(tmem + 128, A(1), B(0), idN256, 1u);  // (1,0) (1,1)
            mma_bf16_ss(tmem + 256, A(2), B(0), idN128, 1u);  // (2,0)
          } else {
            mma_bf16_ss(tmem + 256, A(0), B(2), idN256, f);   // (0,2) (0,3)
            mma_bf16_ss(tmem + 128, A(1), B(0), idN256, 1u);  // (1,0) (1,1)
            mma_bf16_ss(tmem + 384, A(1), B(2), idN128, 1u);  // (1,2)
            mma_bf16_ss(tmem + 256, A(2), B(0), idN256, 1u);  // (2,0) (2,1)
            mma_bf16_ss(tmem + 384, A(3), B(0), idN128, 1u);  // (3,0)
            if (nprod == 13) {
              // order-4 products (1,3), (2,2), (3,1) into the order-3 accumulator
              mma_bf16_ss(tmem + 384, A(1), B(3), idN128, 1u);
              mma_bf16_ss(tmem + 384, A(2), B(2), idN128, 1u);
              mma_bf16_ss(tmem + 384, A(3), B(1), idN128, 1u);
            }
          }
        }
        issued = true;
        if constexpr (CL > 1) mma_commit_mc(empty + s, (uint16_t)peer_mask);
        else mma_commit(empty + s);
        if ((j + 1) % DRAIN_KSTEPS == 0 || j == nK - 1) mma_commit(acc_full);
        if constexpr (RING) mma_commit(emptyB + j % BST);  // this step's D buffer may be refilled
      }
      if (ok && CL > 1) {
        // every peer's commit for the last use of each stage has landed here, so no
        // arrive can reach this CTA's barriers after it exits
        for (int j = (nK > STAGES ? nK - STAGES : 0); j < nK; ++j)
          if (!mbar_wait_cluster(empty + j % STAGES, (uint32_t)((j / STAGES) & 1), abort_flag, g.wait_budget)) break;
      }
      if (!ok) {
        // abort path: let in-flight TMA loads and MMAs finish before the CTA exits
        const long long cleanup = 400000000LL;
        for (int s = 0; s < STAGES; ++s) {
          if (tma_last[s] < 0) continue;
          const long long t0 = clock64();
          while (!mbar_try_wait(wfull + s, (uint32_t)((tma_last[s] / STAGES) & 1)) && clock64() - t0 < cleanup) {
          }
        }
        if (issued) {
          mma_commit(done);
          const long long t0 = clock64();
          while (!mbar_try_wait(done, 0u) && clock64() - t0 < cleanup) {
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == NWORK + 1) {
    // ------------------------------------- cluster copies (1 thread; CL > 1 only)
    if (CL > 1 && lane == 0) {
      constexpr uint32_t ABLK = SLICE_BYTES / CY, BBLK = SLICE_BYTES / CX;
      constexpr uint32_t IN_BYTES = (DT ? 0u : (CX - 1) * NS * BBLK) + (CY - 1) * NS * ABLK;
      const uint32_t sbase = smem_u32(smem);
      for (int j = 0; j < nK; ++j) {
        const int s = j % STAGES;
        if (!mbar_wait(gen + s, (uint32_t)((j / STAGES) & 1), abort_flag, g.wait_budget)) break;
        mbar_arrive_expect_tx(full + s, IN_BYTES);
        const uint32_t st = sbase + (uint32_t)(s * STAGE_STRIDE);
#pragma unroll
        for (int q = 0; q < (DT ? 1 : CX); ++q) {
          if (q == rx) continue;
          const uint32_t peer = (uint32_t)(q + CX * ry);
          const uint32_t bar = mapa(smem_u32(full + s), peer);
#pragma unroll
          for (int v = 0; v < NS; ++v) {
            const uint32_t src = st + A_BYTES + v * SLICE_BYTES + rx * BBLK;
            bulk_copy_to_peer(mapa(src, peer), src, BBLK, bar);
          }
        }
#pragma unroll
        for (int q = 0; q < CY; ++q) {
          if (q == ry) continue;
          const uint32_t peer = (uint32_t)(rx + CX * q);
          const uint32_t bar = mapa(smem_u32(full + s), peer);
#pragma unroll
          for (int u = 0; u < NS; ++u) {
            const uint32_t src = st + u * SLICE_BYTES + ry * ABLK;
            bulk_copy_to_peer(mapa(src, peer), src, ABLK, bar);
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == NWORK + 2) {
    // ------------------------------------- D-slice loads (1 thread; D by TMA only)
    // A k-step's D slices are fetched as soon as their buffer is free (RING: the MMAs of step
    // j - 2 are done; otherwise the stage's), independently of the producers, which may then run
    // up to the full stage depth ahead of the MMAs.
    if (DT && lane == 0) {
      int d_last[BST];
#pragma unroll
      for (int q = 0; q < BST; ++q) d_last[q] = -1;
      for (int j = 0; j < nK; ++j) {
        const int q = j % BST;
        bool free_ = true;
        if (j >= BST) {
          const uint32_t par = (uint32_t)(((j / BST) - 1) & 1);
          if constexpr (RING) free_ = mbar_wait(emptyB + q, par, abort_flag, g.wait_budget);
          else if constexpr (CL > 1) free_ = mbar_wait_cluster(empty + q, par, abort_flag, g.wait_budget);
          else free_ = mbar_wait(empty + q, par, abort_flag, g.wait_budget);
        }
        if (!free_) break;
        uint8_t* dst = RING ? smem + Geo::B_RING + q * B_BYTES : smem + q * STAGE_STRIDE + A_BYTES;
        mbar_arrive_expect_tx(dfull + q, (uint32_t)B_BYTES);
        tma_load_3d(dst, map_d, dfull + q, j * KS, n0, 0);
        d_last[q] = j;
      }
      // no D copy may still be landing when the CTA exits (completed ones return at once)
      const long long cleanup = 400000000LL;
      for (int q = 0; q < BST; ++q) {
        if (d_last[q] < 0) continue;
        const long long t0 = clock64();
        while (!mbar_try_wait(dfull + q, (uint32_t)((d_last[q] / BST) & 1)) && clock64() - t0 < cleanup) {
        }
      }
    }
    __syncwarp();
  } else {
    // -------------------------------------------------- producers and drains
    const int w = warp;
    const bool f16 = g.f16 != 0;
    // slices per operand and accumulator orders the product set uses
    const int nsl = NS == 5 ? 5 : slices_of(g.nprod);
    const int nord = nsl < 4 ? nsl : 4;  // order 4 shares the order-3 accumulator
    // A role (pair rows of i-blocks ry*8/CY .. +8/CY): i-row ai, j-rows
    // jj = jbase + 2t, k-pair kpa; a half-warp writes one full slice row.
    constexpr int TA = 4 / CY;   // j-rows per thread
    const int ai = ry * (8 / CY) + w / (2 * CY);
    const int kpa = lane & 15, jbase = (w % (2 * CY)) * (8 / CY) + (lane >> 4);
    const int gi = I0 + ai;
    float mp[TA];
#pragma unroll
    for (int t = 0; t < TA; ++t) {
      const int gj = J0 + jbase + 2 * t;
      mp[t] = (gi < n && gj < n && gi <= gj) ? g.mult_p[pair_index(n, gi, gj)] : 0.0f;
    }
    // B role (energy rows rx*128/CX .. +128/CX): row rb, k-pairs kpb + 4 (kq0 + t)
    constexpr int RG = 16 / CX;  // 8-row groups formed by this CTA
    constexpr int TB = 4 / CX;   // k-pair groups per thread
    const int rb = rx * (128 / CX) + 8 * (w % RG) + (lane & 7), kpb = lane >> 3;
    const int kq0 = (w / RG) * TB;
    const int eloc = n0 + rb;
    float eh = 1.0e30f, el = 0.0f, me = 0.0f;  // rows past the chunk: finite and zero
    int klo = 0, khi = 0;
    if (eloc < g.ne) {
      const int64_t ge = g.e_begin + eloc;
      eh = g.Eh[ge];
      el = g.El[ge];
      me = g.mult_e[ge];
      klo = g.klo[ge];
      khi = g.khi[ge];
    }
    // swizzled slice offsets of this thread's elements, the same in every k-step
    uint32_t offA[TA], offB[TB];
#pragma unroll
    for (int t = 0; t < TA; ++t) {
      offA[t] = swz(ai * 16 + jbase + 2 * t, 2 * kpa);
      if (!RM_CHECK(offA[t] + 4 <= (uint32_t)SLICE_BYTES)) offA[t] = 0;
    }
#pragma unroll
    for (int t = 0; t < TB; ++t) {
      offB[t] = swz(rb, 2 * (kpb + 4 * (kq0 + t)));
      if (!RM_CHECK(offB[t] + 4 <= (uint32_t)SLICE_BYTES)) offB[t] = 0;
    }
    const uint32_t trow = tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(32 * (w >> 2));
    // running sums of this thread's 32 accumulator cells (pair row 32 (w & 3) + lane, energy
    // columns 32 (w >> 2) + c): high and low parts; with five slices the low parts live in the
    // order-3 columns instead (drain_half), and Vl is unused
    float Vh[32], Vl[NS == 5 ? 1 : 32];
#pragma unroll
    for (int c = 0; c < 32; ++c) Vh[c] = 0.0f;
#pragma unroll
    for (int c = 0; c < (NS == 5 ? 1 : 32); ++c) Vl[c] = 0.0f;
    bool ok = true;
    // Every way out of this loop is taken by whole warps, so that no lane is left at the
    // __syncwarp below while another has gone on to the final barrier: the waits are polled by
    // all lanes of a converged warp in the same instructions (the same barrier phase, abort flag
    // and clock).
    for (int j = 0; j < nK && ok; ++j) {
      const int s = j % STAGES;
      if (j >= STAGES) {
        bool got;
        if constexpr (CL > 1)
          got = mbar_wait_cluster(empty + s, (uint32_t)(((j / STAGES) - 1) & 1), abort_flag, g.wait_budget);
        else got = mbar_wait(empty + s, (uint32_t)(((j / STAGES) - 1) & 1), abort_flag, g.wait_budget);
        if (!got) {
          ok = false;
          break;
        }
      }
      if (!mbar_wait(wfull + s, (uint32_t)((j / STAGES) & 1), abort_flag, g.wait_budget)) {
        ok = false;
        break;
      }
      uint8_t* st = smem + s * STAGE_STRIDE;
      const float* WI = reinterpret_cast<const float*>(st + W_OFF);
      const float* WJ = WI + WI_FLOATS;
      const float* PO = WJ + WJ_FLOATS;
      uint8_t* Ab = st;
      uint8_t* Bb = st + A_BYTES;
      const int ka = 2 * kpa;
      const float2 wih = *reinterpret_cast<const float2*>(WI + (2 * ai) * KS + ka);
      const float2 wil = *reinterpret_cast<const float2*>(WI + (2 * ai + 1) * KS + ka);
#pragma unroll
      for (int t = 0; t < TA; ++t) {
        const int jj = jbase + 2 * t;
        const int k = ka;
        const float2 wjh = *reinterpret_cast<const float2*>(WJ + (2 * jj) * KS + k);
        const float2 wjl = *reinterpret_cast<const float2*>(WJ + (2 * jj + 1) * KS + k);
        float ph0, pl0, ph1, pl1;
        df_mul(wih.x, wil.x, wjh.x, wjl.x, ph0, pl0);
        df_mul(wih.y, wil.y, wjh.y, wjl.y, ph1, pl1);
        if constexpr (NS == 5) {
          float s0[5], s1[5];
          slice5(__fmul_rn(ph0, mp[t]), __fmul_rn(pl0, mp[t]), s0);
          slice5(__fmul_rn(ph1, mp[t]), __fmul_rn(pl1, mp[t]), s1);
#pragma unroll
          for (int u = 0; u < 5; ++u)
            *reinterpret_cast<uint32_t*>(Ab + u * SLICE_BYTES + offA[t]) = pack_bf16x2(s0[u], s1[u]);
        } else {
          float s0[4], s1[4];
          slice4(__fmul_rn(ph0, mp[t]), __fmul_rn(pl0, mp[t]), s0);
          slice4(__fmul_rn(ph1, mp[t]), __fmul_rn(pl1, mp[t]), s1);
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (u < nsl) *reinterpret_cast<uint32_t*>(Ab + u * SLICE_BYTES + offA[t]) = pack_slice(s0[u], s1[u], f16);
        }
      }
      if constexpr (!DT) {
        const int k0 = j * KS;
        // the whole k-step lies outside this energy's near window (and inside the real poles):
        // no per-element test
        const bool all_far = (k0 + KS <= klo || k0 >= khi) && k0 + KS <= g.N;
#pragma unroll
        for (int t = 0; t < TB; ++t) {
          const int k = 2 * (kpb + 4 * (kq0 + t));
          const int kg = k0 + k;
          const float2 ph = *reinterpret_cast<const float2*>(PO + k);
          const float2 pl = *reinterpret_cast<const float2*>(PO + KS + k);
          const bool far0 = all_far || ((kg < klo || kg >= khi) && kg < g.N);
          const bool far1 = all_far || ((kg + 1 < klo || kg + 1 >= khi) && kg + 1 < g.N);
          if constexpr (NS == 5) {
            uint32_t wd[5];
            d_pack5(ph.x, pl.x, ph.y, pl.y, eh, el, far0 ? me : 0.0f, far1 ? me : 0.0f, wd);
#pragma unroll
            for (int v = 0; v < 5; ++v) *reinterpret_cast<uint32_t*>(Bb + v * SLICE_BYTES + offB[t]) = wd[v];
          } else {
            uint32_t wd[4];
            d_pack(ph.x, pl.x, ph.y, pl.y, eh, el, far0 ? me : 0.0f, far1 ? me : 0.0f, f16, wd);
#pragma unroll
            for (int v = 0; v < 4; ++v)
              if (v < nsl) *reinterpret_cast<uint32_t*>(Bb + v * SLICE_BYTES + offB[t]) = wd[v];
          }
        }
      }
      // the MMAs (and, in clusters, the bulk copies) read these slices through the async proxy
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(CL > 1 ? gen + s : full + s);
      if ((j + 1) % DRAIN_KSTEPS == 0 || j == nK - 1) {
        const int d = j / DRAIN_KSTEPS;
        if (!mbar_wait(acc_full, (uint32_t)(d & 1), abort_flag, g.wait_budget)) {
          ok = false;
          break;
        }
        tc_fence_after();
        if constexpr (NS == 5) {
          const bool last = j == nK - 1;
          const int row = 32 * (w & 3) + lane;
          const int pi = I0 + row / 16, pj = J0 + row % 16;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            float lo[16], vh[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) vh[c] = Vh[h * 16 + c];
            drain_half(trow, h, vh, lo);
#pragma unroll
            for (int c = 0; c < 16; ++c) Vh[h * 16 + c] = vh[c];
            if (!last) {
              // the new low parts go back to order 3, and order 2 restarts from zero
              uint32_t r[16], z[16];
#pragma unroll
              for (int c = 0; c < 16; ++c) {
                r[c] = __float_as_uint(lo[c]);
                z[c] = 0u;
              }
              tmem_st16(trow + (uint32_t)(384 + h * 16), r);
              tmem_st16(trow + (uint32_t)(256 + h * 16), z);
            } else if (pi < n && pj < n && pi <= pj) {
              const int64_t np = (int64_t)n * (n + 1) / 2;
              const int64_t p = pair_index(n, pi, pj);
              const double fp = g.f_p[p];
#pragma unroll
              for (int c = 0; c < 16; ++c) {
                const int e = n0 + 32 * (w >> 2) + h * 16 + c;
                if (e < g.ne && RM_CHECK(p >= 0 && p < np))
                  g.R[(int64_t)e * np + p] = ((double)Vh[h * 16 + c] + (double)lo[c]) * fp * g.tau[g.e_begin + e];
              }
            }
          }
          if (!last) tmem_wait_st();
        } else {
          // orders 0-2 by TwoSum into (hi, lo); the order-3 sum is of the size of lo
#pragma unroll
          for (int o = 0; o < 4; ++o) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              uint32_t r[16];
              tmem_ld16(trow + (uint32_t)(o * 128 + h * 16), r);
              tmem_wait_ld();
#pragma unroll
              for (int c = 0; c < 16; ++c) {
                const int i = h * 16 + c;
                // an order the product set leaves unused holds stale TMEM: select it away
                const float x = o < nord ? __uint_as_float(r[c]) : 0.0f;
                if (o < 3) {
                  float sh, se;
                  two_sum(Vh[i], x, sh, se);
                  Vh[i] = sh;
                  Vl[i] = __fadd_rn(Vl[i], se);
                } else {
                  Vl[i] = __fadd_rn(Vl[i], x);
                }
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acc_empty);
      }
    }
    // ------------------------------------------------------------- epilogue
    // (five slices: written by the last drain)
    if constexpr (NS != 5) {
      if (ok) {
        const int row = 32 * (w & 3) + lane;
        const int pi = I0 + row / 16, pj = J0 + row % 16;
        if (pi < n && pj < n && pi <= pj) {
          const int64_t np = (int64_t)n * (n + 1) / 2;
          const int64_t p = pair_index(n, pi, pj);
          const double fp = g.f_p[p];
#pragma unroll
          for (int c = 0; c < 32; ++c) {
            const int e = n0 + 32 * (w >> 2) + c;
            if (e < g.ne && RM_CHECK(p >= 0 && p < np))
              g.R[(int64_t)e * np + p] = ((double)Vh[c] + (double)Vl[c]) * fp * g.tau[g.e_begin + e];
          }
        }
      }
    }
  }
  tc_fence_before();
  if constexpr (CL > 1) cluster_sync();  // no CTA leaves while a peer may still write to it
  else __syncthreads();
  if (warp == NWORK) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
  if (threadIdx.x == 0 && *abort_flag) atomicMax(g.err, (int)RM_ERR_TIMEOUT);
}

template <int NS>
__global__ void __launch_bounds__(NTHREADS, 1)
    polesum_tc_kernel(const __grid_constant__ CUtensorMap map_omega, const __grid_constant__ CUtensorMap map_pol,
                      TCArgs g) {
  extern __shared__ unsigned char smem_raw[];
  const int2 tile = g.tiles[blockIdx.x];
  tc_tile<1, 1, false, NS>(&map_omega, &map_pol, nullptr, g, tile.x * 8, tile.y * 16, blockIdx.y * BN, smem_raw);
}

// Every wave of a plan in one launch: tile list entries (wave, i-block, j-block),
// per-wave arguments and TMA descriptors in global memory; the chunk's energy
// range is shared by all waves.  Launched in clusters of CX x CY CTAs: the tile
// list holds each wave's tiles padded to a multiple of CX, and grid.y is a
// multiple of CY.
template <int CX, int CY, bool DT, int NS>
__global__ void __launch_bounds__(NTHREADS, 1)
    polesum_tc_grouped_kernel(const TCArgs* __restrict__ waves, const CUtensorMap* __restrict__ maps,
                              const int4* __restrict__ tiles, int64_t e_begin, int ne) {
  extern __shared__ unsigned char smem_raw[];
  const int4 t = tiles[blockIdx.x];
  TCArgs g = waves[t.x];
  g.e_begin = e_begin;
  g.ne = ne;
  tc_tile<CX, CY, DT, NS>(maps + 3 * t.x, maps + 3 * t.x + 1, maps + 3 * t.x + 2, g, t.y * 8, t.z * 16,
                          blockIdx.y * BN, smem_raw);
}

// ------------------------------------------------------ 2-SM pole sum (cta_group::2)
//
// The 15-product far sum on a CTA pair whose MMAs run as one: tcgen05.mma.cta_group::2 with
// M = 256 energies (the A operand: each CTA's own 128 energies of D slices, staged by TMA from the
// D-slice kernel's buffer), N = 128 pairs (the B operand: each CTA holds the P slices of the 64
// pairs it forms) and K = 16.  Each SM's tensor core reads its A and its half of B from its own
// shared memory, so per product the B reads halve against the one-SM kernel (6 KB instead of 8 KB
// per SM and K = 16), and no P half travels between the CTAs.  Each CTA's TMEM holds its 128
// energies (lanes) x 128 pairs (columns) per order: order o in columns [128 o, 128 o + 128),
// order 4 sharing order 3, as in the one-SM kernel; pair column c is the pair
// (I0 + c / 16, J0 + c % 16), columns 0-63 formed by the even CTA and 64-127 by the odd one.
//
// Warps (18 per CTA, the same in both CTAs unless stated):
//   0-15  producers: the P slices of the CTA's 64 pairs per k-step; drains and the epilogue
//   16    TMEM allocation (both CTAs, collective); lane 0 of the even CTA issues the MMAs
//   17    lane 0: W-row and D-slice loads, and the readiness of each k-step to the even CTA
// Barriers: wfull / dfull complete on the CTA's own loads, gen on its producers; full (even CTA,
// two arrivals) when both CTAs' operands of a k-step are in place; empty, emptyB and acc_full are
// signalled in both CTAs by the even CTA's commits; acc_empty (even CTA) by the drains of both.
constexpr int PAIR_PSL = 64 * KS * 2;  // 4 KB: one P slice of 64 pairs (64 rows x 64 B)
constexpr int PAIR_NTHREADS = (NWORK + 2) * 32;  // producers + MMA warp + load/readiness warp

template <int PST, int DST>
struct PairGeo {
  static constexpr int D_BYTES = 5 * SLICE_BYTES;  // 40 KB: five D slices of 128 energies
  static constexpr int P_BYTES = 5 * PAIR_PSL;     // 20 KB: five P slices of 64 pairs
  static constexpr int D_OFF = 0;
  static constexpr int P_OFF = DST * D_BYTES;
  static constexpr int W_OFF = P_OFF + PST * P_BYTES;
  static constexpr int BARS_OFF = W_OFF + PST * TX_BYTES;
  static constexpr int NBARS = 4 * PST + 2 * DST + 3;
  static constexpr size_t SMEM = (size_t)BARS_OFF + 1024 + NBARS * 8 + 16;
};
constexpr int PAIR_PST = 4;  // P-slice / W-row stages
constexpr int PAIR_DST = 3;  // D-slice buffers
static_assert(PairGeo<PAIR_PST, PAIR_DST>::SMEM <= 232448, "a CTA's shared memory");
static_assert(TX_BYTES % 128 == 0 && PairGeo<PAIR_PST, PAIR_DST>::W_OFF % 1024 == 0,
              "W rows and slices keep the alignment TMA and the swizzle need");

// the 2-SM kernel runs for 1 x 2 clusters with D by TMA and five slices per operand
bool pair_applies(int cx, int cy, bool dt, int ns, bool pair) { return pair && cx == 1 && cy == 2 && dt && ns == 5; }

template <int PST, int DST>
__device__ __forceinline__ void tc_pair_tile(const CUtensorMap* map_omega, const CUtensorMap* map_pol,
                                             const CUtensorMap* map_d, const TCArgs& g, int I0, int J0, int n0,
                                             unsigned char* smem_raw) {
  using namespace ptx;
  using Geo = PairGeo<PST, DST>;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Geo::BARS_OFF);
  uint64_t* wfull = bars;
  uint64_t* gen = bars + PST;
  uint64_t* full = bars + 2 * PST;
  uint64_t* empty = bars + 3 * PST;
  uint64_t* dfull = bars + 4 * PST;
  uint64_t* emptyB = dfull + DST;
  uint64_t* acc_full = emptyB + DST;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* done = acc_full + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + Geo::NBARS);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nK = g.nK;
  const int n = g.n;
  const uint32_t rank = cluster_ctarank();  // 0: issues the pair's MMAs; 1: its peer
  const bool lead = rank == 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < PST; ++s) {
      mbar_init(wfull + s, 1);
      mbar_init(gen + s, NWORK);
      mbar_init(full + s, 2);  // the readiness arrivals of both CTAs
      mbar_init(empty + s, 1);
    }
    for (int q = 0; q < DST; ++q) {
      mbar_init(dfull + q, 1);
      mbar_init(emptyB + q, 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 2 * NWORK);  // the drain warps of both CTAs
    mbar_init(done, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == NWORK) {
    tmem_alloc_pair(tmem_slot, 512);
    tmem_relinquish_pair();
  }
  tc_fence_before();
  cluster_sync();  // both CTAs' barriers and TMEM exist before any remote arrive or MMA
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == NWORK) {
    // ------------------------------------------- MMA issue (1 thread of the even CTA)
    if (lead && lane == 0) {
      const uint32_t idesc = idesc_bf16_f32(256, 128, false);
      bool ok = true;
      bool issued = false;
      for (int j = 0; j < nK; ++j) {
        const int s = j % PST, q = j % DST;
        if (!mbar_wait_cluster(full + s, (uint32_t)((j / PST) & 1), abort_flag, g.wait_budget)) {
          ok = false;
          break;
        }
        const int d = j / DRAIN_KSTEPS;
        const bool first = (j % DRAIN_KSTEPS) == 0;
        if (first && d > 0 &&
            !mbar_wait_cluster(acc_empty, (uint32_t)((d - 1) & 1), abort_flag, g.wait_budget)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a = smem_u32(smem + Geo::D_OFF + q * Geo::D_BYTES);
        const uint32_t b = smem_u32(smem + Geo::P_OFF + s * Geo::P_BYTES);
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          const uint32_t ko = kk * 32;
          const uint32_t f = (first && kk == 0) ? 0u : 1u;
          // order 3 carries the low parts of the running sums from drain to drain: it starts once
          const uint32_t f3 = (j == 0 && kk == 0) ? 0u : 1u;
          auto A = [&](int v) { return desc_kmajor_sw64(a + v * SLICE_BYTES + ko); };  // D slice v
          auto B = [&](int u) { return desc_kmajor_sw64(b + u * PAIR_PSL + ko); };     // P slice u
          // (u, v) = P slice u times D slice v into order u + v (4 into 3); the first product
          // into each of orders 0-2 of a drain period starts it.  Each order receives its products in
          // the one-SM kernels' sequence, so the inexact FP32 sums of order 3 round alike and
          // the two forms give the same bits.
          mma_bf16_ss_pair(tmem + 0, A(0), B(0), idesc, f);    // (0,0)
          mma_bf16_ss_pair(tmem + 128, A(1), B(0), idesc, f);  // (0,1)
          mma_bf16_ss_pair(tmem + 128, A(0), B(1), idesc, 1u); // (1,0)
          mma_bf16_ss_pair(tmem + 256, A(2), B(0), idesc, f);  // (0,2)
          mma_bf16_ss_pair(tmem + 256, A(1), B(1), idesc, 1u); // (1,1)
          mma_bf16_ss_pair(tmem + 256, A(0), B(2), idesc, 1u); // (2,0)
          mma_bf16_ss_pair(tmem + 384, A(3), B(0), idesc, f3); // (0,3)
          mma_bf16_ss_pair(tmem + 384, A(4), B(0), idesc, 1u); // (0,4)
          mma_bf16_ss_pair(tmem + 384, A(2), B(1), idesc, 1u); // (1,2)
          mma_bf16_ss_pair(tmem + 384, A(3), B(1), idesc, 1u); // (1,3)
          mma_bf16_ss_pair(tmem + 384, A(1), B(2), idesc, 1u); // (2,1)
          mma_bf16_ss_pair(tmem + 384, A(2), B(2), idesc, 1u); // (2,2)
          mma_bf16_ss_pair(tmem + 384, A(0), B(3), idesc, 1u); // (3,0)
          mma_bf16_ss_pair(tmem + 384, A(1), B(3), idesc, 1u); // (3,1)
          mma_bf16_ss_pair(tmem + 384, A(0), B(4), idesc, 1u); // (4,0)
        }
        issued = true;
        mma_commit_pair_mc(empty + s, (uint16_t)3);   // both CTAs may refill this P stage
        mma_commit_pair_mc(emptyB + q, (uint16_t)3);  // and this D buffer
        if ((j + 1) % DRAIN_KSTEPS == 0 || j == nK - 1) mma_commit_pair_mc(acc_full, (uint16_t)3);
      }
      if (!ok && issued) {
        // abort path: the MMAs in flight read both CTAs' shared memory; let them finish
        mma_commit_pair_mc(done, (uint16_t)1);
        const long long t0 = clock64();
        while (!mbar_try_wait(done, 0u) && clock64() - t0 < 400000000LL) {
        }
      }
    }
    __syncwarp();
  } else if (warp == NWORK + 1) {
    // ------------------- W-row and D-slice loads, k-step readiness (1 thread per CTA)
    // Step j is forwarded to the even CTA once this CTA's P slices are formed (gen) and its D
    // slices have landed (dfull); the W rows of step j + PST then refill the stage, and once
    // the MMAs of step j - 1 are done the D slices of step j - 1 + DST refill their buffer:
    // MMA j is then running, so the tensor pipe keeps a step queued while this thread waits,
    // and a D box is issued two MMA steps before its step.
    if (lane == 0) {
      int w_last[PST], d_last[DST];
#pragma unroll
      for (int s = 0; s < PST; ++s) w_last[s] = -1;
#pragma unroll
      for (int q = 0; q < DST; ++q) d_last[q] = -1;
      auto issue_w = [&](int s, int j) {
        float* WI = reinterpret_cast<float*>(smem + Geo::W_OFF + s * TX_BYTES);
        float* WJ = WI + WI_FLOATS;
        float* PO = WJ + WJ_FLOATS;
        mbar_arrive_expect_tx(wfull + s, TX_BYTES);
        const int x = j * KS;
        tma_load_2d(WI, map_omega, wfull + s, x, 2 * I0);
        tma_load_2d(WJ, map_omega, wfull + s, x, 2 * J0);
        tma_load_2d(WJ + 16 * KS, map_omega, wfull + s, x, 2 * J0 + 16);
        tma_load_2d(PO, map_pol, wfull + s, x, 0);
        w_last[s] = j;
      };
      auto issue_d = [&](int j) {
        const int q = j % DST;
        mbar_arrive_expect_tx(dfull + q, (uint32_t)Geo::D_BYTES);
        tma_load_3d(smem + Geo::D_OFF + q * Geo::D_BYTES, map_d, dfull + q, j * KS, n0, 0);
        d_last[q] = j;
      };
      for (int j = 0; j < DST && j < nK; ++j) issue_d(j);
      for (int s = 0; s < PST && s < nK; ++s) issue_w(s, s);
      const uint32_t lead_full = mapa(smem_u32(full), 0u);
      bool ok = true;
      for (int j = 0; j < nK; ++j) {
        const int s = j % PST, q = j % DST;
        // this CTA's P slices of step j are formed (and its W rows read): refill the W rows
        if (!mbar_wait(gen + s, (uint32_t)((j / PST) & 1), abort_flag, g.wait_budget)) {
          ok = false;
          break;
        }
        if (j + PST < nK) issue_w(s, j + PST);
        if (!mbar_wait(dfull + q, (uint32_t)((j / DST) & 1), abort_flag, g.wait_budget)) {
          ok = false;
          break;
        }
        mbar_arrive_cluster(lead_full + (uint32_t)(8 * s));
        const int jd = j - 1 + DST;  // the D slices the MMAs of step j - 1 make room for
        if (j >= 1 && jd < nK) {
          const int qd = (j - 1) % DST;
          if (!mbar_wait_cluster(emptyB + qd, (uint32_t)(((j - 1) / DST) & 1), abort_flag, g.wait_budget)) {
            ok = false;
            break;
          }
          issue_d(jd);
        }
      }
      if (ok) {
        // the even CTA's commits for the last uses of every stage and D buffer have landed
        // here, so none can reach this CTA's barriers after it exits
        for (int j = (nK > PST ? nK - PST : 0); j < nK; ++j)
          if (!mbar_wait_cluster(empty + j % PST, (uint32_t)((j / PST) & 1), abort_flag, g.wait_budget)) break;
        for (int j = (nK > DST ? nK - DST : 0); j < nK; ++j)
          if (!mbar_wait_cluster(emptyB + j % DST, (uint32_t)((j / DST) & 1), abort_flag, g.wait_budget)) break;
      }
      // no W or D copy may still be landing when the CTA exits (completed ones return at once)
      for (int s = 0; s < PST; ++s) {
        if (w_last[s] < 0) continue;
        const long long t0 = clock64();
        while (!mbar_try_wait(wfull + s, (uint32_t)((w_last[s] / PST) & 1)) && clock64() - t0 < 400000000LL) {
        }
      }
      for (int q = 0; q < DST; ++q) {
        if (d_last[q] < 0) continue;
        const long long t0 = clock64();
        while (!mbar_try_wait(dfull + q, (uint32_t)((d_last[q] / DST) & 1)) && clock64() - t0 < 400000000LL) {
        }
      }
    }
    __syncwarp();
  } else {
    // -------------------------------------------------- producers and drains
    const int w = warp;
    // P rows of this CTA's 64 pairs: tile i-channel ai = 4 rank + w / 4, j-channels
    // jj = jbase + 2t (t = 0, 1), pole pair kpa; a half-warp writes one full slice row
    const int ail = w >> 2;
    const int ai = 4 * (int)rank + ail;
    const int kpa = lane & 15, jbase = 4 * (w & 3) + (lane >> 4);
    const int gi = I0 + ai;
    float mp[2];
    uint32_t offP[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int jj = jbase + 2 * t;
      const int gj = J0 + jj;
      mp[t] = (gi < n && gj < n && gi <= gj) ? g.mult_p[pair_index(n, gi, gj)] : 0.0f;
      offP[t] = swz(ail * 16 + jj, 2 * kpa);
      if (!RM_CHECK(offP[t] + 4 <= (uint32_t)PAIR_PSL)) offP[t] = 0;
    }
    const uint32_t trow = tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(32 * (w >> 2));
    const uint32_t lead_acc_empty = mapa(smem_u32(acc_empty), 0u);
    // high parts of the running sums of this thread's 32 accumulator cells (lane = energy row
    // 32 (w & 3) + lane, columns 32 (w >> 2) + c); the low parts live in the order-3 columns
    float Vh[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) Vh[c] = 0.0f;
    bool ok = true;
    // A drain period's accumulators are read LAG k-steps after its last one is formed, so that
    // the operands of the next period's first steps are in place when the MMAs resume.  Forming
    // step j needs the MMAs of step j - PST done, which needed the drain of the period ending at
    // step j - PST - 1 at the latest, run in iteration j - 2: LAG = PST - 1 cannot deadlock.
    constexpr int LAG = PST - 1;
    // every way out of this loop is taken by whole warps (converged polling of the same waits)
    for (int j = 0; j < nK + LAG && ok; ++j) {
      const int s = j % PST;
      if (j < nK) {
        if (j >= PST &&
            !mbar_wait_cluster(empty + s, (uint32_t)(((j / PST) - 1) & 1), abort_flag, g.wait_budget)) {
          ok = false;
          break;
        }
        if (!mbar_wait(wfull + s, (uint32_t)((j / PST) & 1), abort_flag, g.wait_budget)) {
          ok = false;
          break;
        }
        const float* WI = reinterpret_cast<const float*>(smem + Geo::W_OFF + s * TX_BYTES);
        const float* WJ = WI + WI_FLOATS;
        uint8_t* Pb = smem + Geo::P_OFF + s * Geo::P_BYTES;
        const int ka = 2 * kpa;
        const float2 wih = *reinterpret_cast<const float2*>(WI + (2 * ai) * KS + ka);
        const float2 wil = *reinterpret_cast<const float2*>(WI + (2 * ai + 1) * KS + ka);
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          const int jj = jbase + 2 * t;
          const float2 wjh = *reinterpret_cast<const float2*>(WJ + (2 * jj) * KS + ka);
          const float2 wjl = *reinterpret_cast<const float2*>(WJ + (2 * jj + 1) * KS + ka);
          float ph0, pl0, ph1, pl1;
          df_mul(wih.x, wil.x, wjh.x, wjl.x, ph0, pl0);
          df_mul(wih.y, wil.y, wjh.y, wjl.y, ph1, pl1);
          float s0[5], s1[5];
          slice5(__fmul_rn(ph0, mp[t]), __fmul_rn(pl0, mp[t]), s0);
          slice5(__fmul_rn(ph1, mp[t]), __fmul_rn(pl1, mp[t]), s1);
#pragma unroll
          for (int u = 0; u < 5; ++u)
            *reinterpret_cast<uint32_t*>(Pb + u * PAIR_PSL + offP[t]) = pack_bf16x2(s0[u], s1[u]);
        }
        // the tensor cores read these slices through the async proxy
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(gen + s);
      }
      const int je = j - LAG;  // last k-step of the drain period read in this iteration, if any
      if (je >= 0 && ((je + 1) % DRAIN_KSTEPS == 0 || je == nK - 1)) {
        const int d = je / DRAIN_KSTEPS;
        if (!mbar_wait_cluster(acc_full, (uint32_t)(d & 1), abort_flag, g.wait_budget)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const bool last = je == nK - 1;
        const int e = n0 + 32 * (w & 3) + lane;  // this thread's energy row
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          // orders 0-2 into the high parts by TwoSum; their errors and the order-3 column (the
          // previous low part plus this period's order-3 and order-4 products) make the new low
          // part, which goes back to the order-3 column, or with the last period to R
          float lo[16], vh[16];
#pragma unroll
          for (int c = 0; c < 16; ++c) vh[c] = Vh[h * 16 + c];
          drain_half(trow, h, vh, lo);
#pragma unroll
          for (int c = 0; c < 16; ++c) Vh[h * 16 + c] = vh[c];
          if (!last) {
            uint32_t r[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) r[c] = __float_as_uint(lo[c]);
            tmem_st16(trow + (uint32_t)(384 + h * 16), r);
          } else if (e < g.ne) {
            // cells h * 16 + c are the pairs (I0 + 2 (w >> 2) + h, J0 + c)
            const int64_t np = (int64_t)n * (n + 1) / 2;
            const int pi = I0 + 2 * (w >> 2) + h;
            const double te = g.tau[g.e_begin + e];
            double* Re = g.R + (int64_t)e * np;
#pragma unroll
            for (int c = 0; c < 16; ++c) {
              const int pj = J0 + c;
              if (pi < n && pj < n && pi <= pj) {
                const int64_t p = pair_index(n, pi, pj);
                if (RM_CHECK(p >= 0 && p < np)) Re[p] = ((double)Vh[h * 16 + c] + (double)lo[c]) * g.f_p[p] * te;
              }
            }
          }
        }
        if (!last) tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(lead_acc_empty);
      }
    }
  }
  tc_fence_before();
  cluster_sync();  // neither CTA leaves while the pair's MMAs or the peer's arrivals may reach it
  if (warp == NWORK) {
    tc_fence_after();
    tmem_dealloc_pair(tmem, 512);
  }
  if (threadIdx.x == 0 && *abort_flag) atomicMax(g.err, (int)RM_ERR_TIMEOUT);
}

// Every wave of a plan in one launch.  A CTA pair is the two CTAs of a 2 x 1 x 1 cluster (the
// pairing of cta_group::2 runs along the cluster's x): grid (2, tiles, energy-tile pairs), so that
// blockIdx.x is the CTA's rank in its pair, blockIdx.y its pair tile and blockIdx.z the pair of
// energy tiles; consecutive clusters hold consecutive pair tiles of the same energies, as in the
// one-SM launch, and share their D slices in L2.
__global__ void __launch_bounds__(PAIR_NTHREADS, 1)
    polesum_tc_pair_kernel(const TCArgs* __restrict__ waves, const CUtensorMap* __restrict__ maps,
                           const int4* __restrict__ tiles, int64_t e_begin, int ne) {
  extern __shared__ unsigned char smem_raw[];
  const int4 t = tiles[blockIdx.y];
  TCArgs g = waves[t.x];
  g.e_begin = e_begin;
  g.ne = ne;
  tc_pair_tile<PAIR_PST, PAIR_DST>(maps + 3 * t.x, maps + 3 * t.x + 1, maps + 3 * t.x + 2, g, t.y * 8, t.z * 16,
                                   (int)(2 * blockIdx.z + blockIdx.x) * BN, smem_raw);
}

// ------------------------------------------------------------ preparation
// sigma_i = 2^ceil(log2 max_k |w_ik|); w_ik / sigma_i as FP32 hi (row 2i) + lo (row 2i+1)
__global__ void prep_omega_kernel(const double* __restrict__ W, int n, int N, int Npad, double* __restrict__ sigma,
                                  float* __restrict__ omega) {
  const int i = blockIdx.x;
  __shared__ double red[32];
  double m = 0.0;
  for (int k = threadIdx.x; k < N; k += blockDim.x) m = fmax(m, fabs(W[(int64_t)i * Npad + k]));
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) mm = fmax(mm, red[q]);
    int ex = 0;
    double sg = 1.0;
    if (mm > 0.0) {
      frexp(mm, &ex);  // mm = f 2^ex, f in [0.5, 1)
      sg = ldexp(1.0, ex);
    }
    red[0] = sg;
    sigma[i] = sg;
  }
  __syncthreads();
  const double inv = 1.0 / red[0];  // power of two: exact
  for (int k = threadIdx.x; k < Npad; k += blockDim.x) {
    float h = 0.0f, l = 0.0f;
    if (k < N) {
      const double v = W[(int64_t)i * Npad + k] * inv;
      h = (float)v;
      l = (float)(v - (double)h);
    }
    omega[(int64_t)(2 * i) * Npad + k] = h;
    omega[(int64_t)(2 * i + 1) * Npad + k] = l;
  }
}

__global__ void prep_pol_kernel(const double* __restrict__ poles, int N, int Npad, float* __restrict__ pol) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Npad) return;
  float h = 0.0f, l = 0.0f;
  if (k < N) {
    h = (float)poles[k];
    l = (float)(poles[k] - (double)h);
  }
  pol[k] = h;
  pol[Npad + k] = l;
}

// per pair: 2^e_p with max_k |fl(omega_i omega_j)| 2^e_p <= 1; mult_p = 2^(e_p+8),
// f_p = sigma_i sigma_j 2^-e_p 2^-16 / (2a)  (2^-16 undoes the two 2^8 scales)
__global__ void prep_pairs_kernel(const float* __restrict__ omega, const double* __restrict__ sigma, int n, int N,
                                  int Npad, double inv2a, float* __restrict__ mult_p, double* __restrict__ f_p) {
  const int64_t np = (int64_t)n * (n + 1) / 2;
  const int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (p >= np) return;
  const int lane = threadIdx.x & 31;
  // unpack p -> (i, j)
  const double b = 2.0 * n + 1.0;
  int i = (int)floor((b - sqrt(b * b - 8.0 * (double)p)) * 0.5);
  if (i < 0) i = 0;
  while (i > 0 && pair_index(n, i, i) > p) --i;
  while (i + 1 < n && pair_index(n, i + 1, i + 1) <= p) ++i;
  const int j = i + (int)(p - pair_index(n, i, i));
  const float* wi = omega + (int64_t)(2 * i) * Npad;
  const float* wj = omega + (int64_t)(2 * j) * Npad;
  float m = 0.0f;
  for (int k = lane; k < N; k += 32) m = fmaxf(m, fabsf(__fmul_rn(wi[k], wj[k])));
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, off));
  if (lane == 0) {
    if (m == 0.0f) {
      mult_p[p] = 0.0f;
      f_p[p] = 0.0;
    } else {
      int ex = 0;
      frexpf(m, &ex);  // m = f 2^ex, f in [0.5, 1)
      int ep = -ex;
      if (ep > 110) ep = 110;
      mult_p[p] = ldexpf(1.0f, ep + 8);
      f_p[p] = ldexp(sigma[i] * sigma[j], -ep - 16) * inv2a;
    }
  }
}

__device__ inline int lower_bound_d(const double* v, int m, double x) {
  int lo = 0, hi = m;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (v[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}
__device__ inline int upper_bound_d(const double* v, int m, double x) {
  int lo = 0, hi = m;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (v[mid] <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// per energy: near window [klo, khi) = {k : |E_k - E| < delta}, the power-of-two
// scale tau >= max over far poles of |1/(E_k - E)|, and E split into FP32 hi + lo
__global__ void prep_energy_split_kernel(const double* __restrict__ E, int64_t n_e, const double* __restrict__ poles,
                                         int N, double delta, int32_t* __restrict__ klo, int32_t* __restrict__ khi,
                                         double* __restrict__ tau, float* __restrict__ mult_e, float* __restrict__ Eh,
                                         float* __restrict__ El) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_e) return;
  const double x = E[e];
  const int lo = upper_bound_d(poles, N, x - delta);  // first E_k > x - delta
  const int hi = lower_bound_d(poles, N, x + delta);  // first E_k >= x + delta
  double dmin = INFINITY;
  if (lo > 0) dmin = fmin(dmin, x - poles[lo - 1]);
  if (hi < N) dmin = fmin(dmin, poles[hi] - x);
  double t = 1.0;
  if (dmin < INFINITY && dmin > 0.0) {
    int ex = 0;
    frexp(1.001 / dmin, &ex);
    t = ldexp(1.0, ex);
  }
  klo[e] = lo;
  khi[e] = hi;
  tau[e] = t;
  mult_e[e] = (float)(256.0 / t);
  const float h = (float)x;
  Eh[e] = h;
  El[e] = (float)(x - (double)h);
}

// ---------------------------------------------------------- D-slice kernel
// The D slices of a chunk for the tensor-core pole sum (shapes with cluster_x = 1): row e
// (chunk-relative energy) of slice v at D[(v rows + e) Npad / 2 + k / 2], two poles per word, the
// same values the producers would form (d_pack); rows past the chunk's energies are zero.
struct DSliceWave {
  const float* pol;     // [2][Npad] poles, FP32 hi row then lo row
  const float* Eh;      // per absolute energy: FP32 hi, lo, D scale, near window [klo, khi)
  const float* El;
  const float* mult_e;
  const int32_t* klo;
  const int32_t* khi;
  uint32_t* D;          // [ns][rows][Npad / 2]
  int N, Npad, rows, f16;
  int ns;               // slices per operand: 4, or 5 for the 15-product set
};

__global__ void __launch_bounds__(256) dslice_grouped_kernel(const DSliceWave* __restrict__ waves, int64_t e_begin,
                                                             int ne) {
  const DSliceWave w = waves[blockIdx.y];
  const int e = blockIdx.x;  // chunk-relative energy row
  if (e >= w.rows) return;
  float eh = 1.0e30f, el = 0.0f, me = 0.0f;
  int klo = 0, khi = 0;
  if (e < ne) {
    const int64_t ge = e_begin + e;
    eh = w.Eh[ge];
    el = w.El[ge];
    me = w.mult_e[ge];
    klo = w.klo[ge];
    khi = w.khi[ge];
  }
  const int np2 = w.Npad >> 1;
  const int64_t plane = (int64_t)w.rows * np2;
  uint32_t* row = w.D + (int64_t)e * np2;
  if (!RM_CHECK(np2 * 2 == w.Npad && w.N <= w.Npad)) return;
  for (int kp = threadIdx.x; kp < np2; kp += blockDim.x) {
    const int k = 2 * kp;
    const float2 ph = *reinterpret_cast<const float2*>(w.pol + k);
    const float2 pl = *reinterpret_cast<const float2*>(w.pol + w.Npad + k);
    const bool far0 = (k < klo || k >= khi) && k < w.N;
    const bool far1 = (k + 1 < klo || k + 1 >= khi) && k + 1 < w.N;
    if (w.ns == 5) {
      uint32_t wd[5];
      d_pack5(ph.x, pl.x, ph.y, pl.y, eh, el, far0 ? me : 0.0f, far1 ? me : 0.0f, wd);
#pragma unroll
      for (int v = 0; v < 5; ++v) row[v * plane + kp] = wd[v];
    } else {
      uint32_t wd[4];
      d_pack(ph.x, pl.x, ph.y, pl.y, eh, el, far0 ? me : 0.0f, far1 ? me : 0.0f, w.f16 != 0, wd);
#pragma unroll
      for (int v = 0; v < 4; ++v) row[v * plane + kp] = wd[v];
    }
  }
}

// ------------------------------------------------------- near-pole window
constexpr int NEB = 16;   // energies per CTA (they share each pair's products w_ik w_jk)
constexpr int NKP = 32;   // poles per staged piece
constexpr int NNT = 256;  // threads

struct NearWave {
  const double* W;
  const double* poles;
  const double* E;
  const int32_t* klo;
  const int32_t* khi;
  double* R;  // chunk R buffer of this wave
  double inv2a;
  int n, Npad;
};

__device__ __forceinline__ void near_block(const double* __restrict__ W, int n, int Npad,
                                           const double* __restrict__ poles, const double* __restrict__ E,
                                           const int32_t* __restrict__ klo, const int32_t* __restrict__ khi, int ne,
                                           double inv2a, int splits, double* __restrict__ R, int e0, double* nsm) {
  double* Ws = nsm;                       // [n][NKP + 1]
  double* Dm = Ws + (size_t)n * (NKP + 1);  // [NEB][NKP]
  const int e1 = min(ne, e0 + NEB);
  if (e0 >= ne) return;
  const int64_t np = (int64_t)n * (n + 1) / 2;
  const int64_t pb = np * blockIdx.y / splits, pe = np * (blockIdx.y + 1) / splits;
  const int Klo = klo[e0], Khi = khi[e1 - 1];
  const int t = threadIdx.x;
  for (int Ks = Klo; Ks < Khi; Ks += NKP) {
    // groups of 8 poles that hold window poles (the last piece of a window is usually partial)
    const int ng = (min(NKP, Khi - Ks) + 7) >> 3;
    for (int idx = t; idx < n * NKP; idx += NNT) {
      const int i = idx / NKP, kk = idx % NKP;
      Ws[i * (NKP + 1) + kk] = (Ks + kk < Khi && RM_CHECK(Ks + kk < Npad)) ? W[(int64_t)i * Npad + Ks + kk] : 0.0;
    }
    for (int idx = t; idx < NEB * NKP; idx += NNT) {
      const int e = idx / NKP, kk = idx % NKP;
      const int k = Ks + kk;
      double v = 0.0;
      if (e0 + e < e1 && k >= klo[e0 + e] && k < khi[e0 + e]) v = inv2a / (poles[k] - E[e0 + e]);
      Dm[idx] = v;
    }
    __syncthreads();
    // this thread's first pair
    int64_t p = pb + t;
    if (p < pe) {
      const double b = 2.0 * n + 1.0;
      int i = (int)floor((b - sqrt(b * b - 8.0 * (double)p)) * 0.5);
      if (i < 0) i = 0;
      while (i > 0 && pair_index(n, i, i) > p) --i;
      while (i + 1 < n && pair_index(n, i + 1, i + 1) <= p) ++i;
      int j = i + (int)(p - pair_index(n, i, i));
      for (; p < pe; p += NNT) {
        double P[NKP];
#pragma unroll
        for (int g8 = 0; g8 < NKP / 8; ++g8)
          if (g8 < ng) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int kk = 8 * g8 + q;
              P[kk] = Ws[i * (NKP + 1) + kk] * Ws[j * (NKP + 1) + kk];
            }
          }
        for (int e = 0; e < e1 - e0; ++e) {
          double acc = 0.0;
#pragma unroll
          for (int g8 = 0; g8 < NKP / 8; ++g8)
            if (g8 < ng) {
#pragma unroll
              for (int q = 0; q < 8; ++q) acc = fma(P[8 * g8 + q], Dm[e * NKP + 8 * g8 + q], acc);
            }
          if (RM_CHECK(e0 + e < ne && p < np)) R[(int64_t)(e0 + e) * np + p] += acc;
        }
        j += NNT;
        while (j >= n && i < n - 1) {
          ++i;
          j = j - n + i;
        }
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(NNT) near_kernel(const double* __restrict__ W, int n, int Npad,
                                                   const double* __restrict__ poles, const double* __restrict__ E,
                                                   const int32_t* __restrict__ klo, const int32_t* __restrict__ khi,
                                                   int ne, double inv2a, int splits, double* __restrict__ R) {
  extern __shared__ double nsm[];
  near_block(W, n, Npad, poles, E, klo, khi, ne, inv2a, splits, R, blockIdx.x * NEB, nsm);
}

// All waves: job (wave, first energy of the block); energies are chunk-relative.
__global__ void __launch_bounds__(NNT) near_grouped_kernel(const NearWave* __restrict__ waves,
                                                           const int2* __restrict__ jobs, int64_t e_begin, int ne,
                                                           int splits) {
  extern __shared__ double nsm[];
  const int2 jb = jobs[blockIdx.x];
  const NearWave w = waves[jb.x];
  near_block(w.W, w.n, w.Npad, w.poles, w.E + e_begin, w.klo + e_begin, w.khi + e_begin, ne, w.inv2a, splits, w.R,
             jb.y, nsm);
}

PFN_cuTensorMapEncodeTiled_v12000 get_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* ptr = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }
  return fn;
}

bool encode_2d_f32(CUtensorMap* map, const float* base, uint64_t cols, uint64_t rows, uint32_t box_cols,
                   uint32_t box_rows) {
  auto enc = get_encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * sizeof(float)};
  cuuint32_t box[2] = {box_cols, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

size_t polesum_tc_smem_bytes() {
  size_t m = TcGeo<4>::SMEM;
  if (TcGeo<5>::SMEM > m) m = TcGeo<5>::SMEM;
  if (TcGeo<5, true>::SMEM > m) m = TcGeo<5, true>::SMEM;
  if (PairGeo<PAIR_PST, PAIR_DST>::SMEM > m) m = PairGeo<PAIR_PST, PAIR_DST>::SMEM;
  return m;
}
int polesum_slice_planes(int nprod) { return slices_of(nprod) == 5 ? 5 : 4; }
bool polesum_pair_runs(const Plan& p) {
  return pair_applies(p.grp.tc_cx, p.grp.tc_cy, p.grp.dt(), polesum_slice_planes(p.slices), p.grp.tc_pair) &&
         p.prec == RM_PREC_SPLIT_BF16;
}

std::vector<int2> split_tiles(int n) {
  std::vector<int2> t;
  const int nbi = (n + 7) / 8, nbj = (n + 15) / 16;
  for (int I = 0; I < nbi; ++I)
    for (int J = 0; J < nbj; ++J)
      if (16 * J + 15 >= 8 * I) t.push_back(make_int2(I, J));
  return t;
}

cudaError_t split_prepare(const Plan& p, WaveDev& w, cudaStream_t s) {
  SplitDev& sd = w.split;
  // every row of the pole-sum operand (the dipole row, when present, is row 0)
  prep_omega_kernel<<<w.nR, 256, 0, s>>>(w.W, w.nR, w.N, w.Npad, sd.sigma, sd.omega);
  prep_pol_kernel<<<(w.Npad + 255) / 256, 256, 0, s>>>(w.poles, w.N, w.Npad, sd.pol);
  const int64_t np = w.npR();
  prep_pairs_kernel<<<(unsigned)((np + 7) / 8), 256, 0, s>>>(sd.omega, sd.sigma, w.nR, w.N, w.Npad, 1.0 / (2.0 * w.a),
                                                             sd.mult_p, sd.f_p);
  if (p.n_e > 0)
    prep_energy_split_kernel<<<(unsigned)((p.n_e + 255) / 256), 256, 0, s>>>(
        w.E, p.n_e, w.poles, w.N, p.delta, sd.klo, sd.khi, sd.tau, sd.mult_e, sd.Eh, sd.El);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (!encode_2d_f32(&sd.map_omega, sd.omega, (uint64_t)w.Npad, (uint64_t)(2 * w.nR), KS, 16))
    return cudaErrorInvalidValue;
  if (!encode_2d_f32(&sd.map_pol, sd.pol, (uint64_t)w.Npad, 2, KS, 2)) return cudaErrorInvalidValue;
  return cudaSuccess;
}

cudaError_t launch_polesum_split(const Plan& p, const WaveDev& w, int64_t e0, int ne, double* R, cudaStream_t s) {
  if (ne <= 0) return cudaSuccess;
  const SplitDev& sd = w.split;
  TCArgs g;
  g.mult_p = sd.mult_p;
  g.f_p = sd.f_p;
  g.klo = sd.klo;
  g.khi = sd.khi;
  g.tau = sd.tau;
  g.mult_e = sd.mult_e;
  g.Eh = sd.Eh;
  g.El = sd.El;
  g.tiles = sd.tiles;
  g.n = w.nR;
  g.N = w.N;
  g.nK = w.Npad / KS;
  g.f16 = p.prec == RM_PREC_SPLIT_FP16 ? 1 : 0;
  g.nprod = p.slices;
  g.wait_budget = p.fault_wait > 0 ? p.fault_wait : WAIT_BUDGET;  // this launch runs unclustered
  g.e_begin = e0;
  g.ne = ne;
  g.R = R;
  g.err = p.err_word;
  dim3 grid(sd.n_tiles, (ne + BN - 1) / BN);
  if (slices_of(p.slices) == 5) {
    cudaError_t err = cudaFuncSetAttribute(polesum_tc_kernel<5>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)TcGeo<5>::SMEM);
    if (err != cudaSuccess) return err;
    polesum_tc_kernel<5><<<grid, NTHREADS, TcGeo<5>::SMEM, s>>>(sd.map_omega, sd.map_pol, g);
  } else {
    cudaError_t err = cudaFuncSetAttribute(polesum_tc_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)TcGeo<4>::SMEM);
    if (err != cudaSuccess) return err;
    polesum_tc_kernel<4><<<grid, NTHREADS, TcGeo<4>::SMEM, s>>>(sd.map_omega, sd.map_pol, g);
  }
  return cudaGetLastError();
}

size_t near_smem_bytes(int n) { return ((size_t)n * (NKP + 1) + NEB * NKP) * sizeof(double); }

cudaError_t launch_near(const Plan& p, const WaveDev& w, int64_t e0, int ne, double* R, cudaStream_t s) {
  if (ne <= 0) return cudaSuccess;
  const size_t smem = near_smem_bytes(w.nR);
  cudaError_t err = cudaFuncSetAttribute(near_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  const int blocks = (ne + NEB - 1) / NEB;
  int splits = (2 * p.sm_count + blocks - 1) / blocks;
  if (splits < 1) splits = 1;
  if (splits > 64) splits = 64;
  dim3 grid(blocks, splits);
  near_kernel<<<grid, NNT, smem, s>>>(w.W, w.nR, w.Npad, w.poles, w.E + e0, w.split.klo + e0, w.split.khi + e0, ne,
                                      1.0 / (2.0 * w.a), splits, R);
  return cudaGetLastError();
}

namespace {

using GroupedFn = void (*)(const TCArgs*, const CUtensorMap*, const int4*, int64_t, int);

template <int NS>
GroupedFn grouped_fn_ns(int cx, int cy, bool dt) {
  if (dt) {
    if (cx == 1 && cy == 1) return polesum_tc_grouped_kernel<1, 1, true, NS>;
    if (cx == 1 && cy == 2) return polesum_tc_grouped_kernel<1, 2, true, NS>;
    if (cx == 1 && cy == 4) return polesum_tc_grouped_kernel<1, 4, true, NS>;
    return nullptr;
  }
  if (cx == 1 && cy == 1) return polesum_tc_grouped_kernel<1, 1, false, NS>;
  if (cx == 2 && cy == 1) return polesum_tc_grouped_kernel<2, 1, false, NS>;
  if (cx == 4 && cy == 1) return polesum_tc_grouped_kernel<4, 1, false, NS>;
  if (cx == 1 && cy == 2) return polesum_tc_grouped_kernel<1, 2, false, NS>;
  if (cx == 2 && cy == 2) return polesum_tc_grouped_kernel<2, 2, false, NS>;
  if (cx == 4 && cy == 2) return polesum_tc_grouped_kernel<4, 2, false, NS>;
  if (cx == 2 && cy == 4) return polesum_tc_grouped_kernel<2, 4, false, NS>;
  if (cx == 1 && cy == 4) return polesum_tc_grouped_kernel<1, 4, false, NS>;
  return nullptr;
}

// the grouped kernel for a cluster shape, D staging, slice count (4 or 5 per operand) and MMA form
GroupedFn grouped_fn(int cx, int cy, bool dt, int ns, bool pair) {
  if (pair_applies(cx, cy, dt, ns, pair)) return polesum_tc_pair_kernel;
  return ns == 5 ? grouped_fn_ns<5>(cx, cy, dt) : grouped_fn_ns<4>(cx, cy, dt);
}

// dynamic shared memory of a grouped kernel (five slices with D by TMA: the D ring)
size_t grouped_smem(int cx, int cy, bool dt, int ns, bool pair) {
  if (pair_applies(cx, cy, dt, ns, pair)) return PairGeo<PAIR_PST, PAIR_DST>::SMEM;
  return ns == 5 ? (dt ? TcGeo<5, true>::SMEM : TcGeo<5>::SMEM) : TcGeo<4>::SMEM;
}

cudaError_t set_tc_smem() {
  const int shapes[8][2] = {{1, 1}, {2, 1}, {4, 1}, {1, 2}, {2, 2}, {4, 2}, {2, 4}, {1, 4}};
  for (int ns = 4; ns <= 5; ++ns)
    for (int dt = 0; dt < 2; ++dt)
      for (int pair = 0; pair < 2; ++pair)
        for (const auto& sh : shapes) {
          if (pair && !pair_applies(sh[0], sh[1], dt != 0, ns, true)) continue;
          GroupedFn fn = grouped_fn(sh[0], sh[1], dt != 0, ns, pair != 0);
          if (!fn) continue;
          cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)grouped_smem(sh[0], sh[1], dt != 0, ns, pair != 0));
          if (err != cudaSuccess) return err;
        }
  return cudaSuccess;
}

// 16-bit [ns][rows][Npad] array of D slices, 32-pole x 128-energy x ns-slice boxes in the 64-byte
// swizzle the MMA descriptors expect (the producers' layout, swz)
bool encode_3d_d(CUtensorMap* map, const uint32_t* base, uint64_t npad, uint64_t rows, int ns) {
  auto enc = get_encoder();
  if (!enc) return false;
  cuuint64_t dims[3] = {npad, rows, (cuuint64_t)ns};
  cuuint64_t strides[2] = {npad * 2, rows * npad * 2};
  cuuint32_t box[3] = {(cuuint32_t)KS, (cuuint32_t)BN, (cuuint32_t)ns};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<uint32_t*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

cudaError_t group_setup_split(Plan& p) {
  GroupDev& G = p.grp;
  const int W = p.n_waves;
  std::vector<TCArgs> tw(W);
  std::vector<NearWave> nw(W);
  std::vector<CUtensorMap> maps(3 * W);
  std::vector<DSliceWave> dw(W);
  std::vector<int4> tiles;
  std::vector<int2> jobs;
  for (int g = 0; g < W; ++g) {
    const WaveDev& w = p.waves[g];
    const SplitDev& sd = w.split;
    TCArgs a;
    a.mult_p = sd.mult_p;
    a.f_p = sd.f_p;
    a.klo = sd.klo;
    a.khi = sd.khi;
    a.tau = sd.tau;
    a.mult_e = sd.mult_e;
    a.Eh = sd.Eh;
    a.El = sd.El;
    a.tiles = nullptr;
    a.n = w.nR;
    a.N = w.N;
    a.nK = w.Npad / KS;
    a.f16 = p.prec == RM_PREC_SPLIT_FP16 ? 1 : 0;
    a.nprod = p.slices;
    // the test hook that shortens the waits applies to unclustered launches only: there no
    // other CTA's copies or commits can still be arriving when an aborted tile exits
    a.wait_budget = (p.fault_wait > 0 && G.tc_cx * G.tc_cy == 1) ? p.fault_wait : WAIT_BUDGET;
    a.e_begin = 0;
    a.ne = 0;
    a.R = G.R[g];
    a.err = p.err_word;
    tw[g] = a;
    maps[3 * g] = sd.map_omega;
    maps[3 * g + 1] = sd.map_pol;
    std::memset(&maps[3 * g + 2], 0, sizeof(CUtensorMap));
    if (G.d_rows > 0 && G.D[g]) {
      if (!encode_3d_d(&maps[3 * g + 2], G.D[g], (uint64_t)w.Npad, (uint64_t)G.d_rows, polesum_slice_planes(p.slices)))
        return cudaErrorInvalidValue;
    }
    dw[g] = DSliceWave{sd.pol, sd.Eh, sd.El, sd.mult_e, sd.klo, sd.khi, G.D[g], w.N, w.Npad, G.d_rows,
                       p.prec == RM_PREC_SPLIT_FP16 ? 1 : 0, polesum_slice_planes(p.slices)};
    const std::vector<int2> wt = split_tiles(w.nR);
    for (const int2& t : wt) tiles.push_back(make_int4(g, t.x, t.y, w.Npad / KS));
    // pad to a multiple of the cluster width with empty tiles (i-block past the last channel)
    for (size_t q = wt.size(); q % G.tc_cx != 0; ++q) tiles.push_back(make_int4(g, (w.nR + 7) / 8, 0, w.Npad / KS));
    nw[g] = NearWave{w.W, w.poles, w.E, sd.klo, sd.khi, G.R[g], 1.0 / (2.0 * w.a), w.nR, w.Npad};
    for (int e = 0; e < G.chunk; e += NEB) jobs.push_back(make_int2(g, e));
  }
  // longest K loop first, so the last wave of CTAs holds the short tiles; the sort is
  // stable and each wave's block is a multiple of the cluster width, so every
  // cluster holds tiles of one wave
  std::stable_sort(tiles.begin(), tiles.end(), [](const int4& x, const int4& y) { return x.w > y.w; });
  int splits = (2 * p.sm_count + (int)jobs.size() - 1) / (int)jobs.size();
  G.near_splits = splits < 1 ? 1 : (splits > 64 ? 64 : splits);
  cudaError_t err;
  auto ensure = [&](void** ptr, size_t bytes, size_t old_bytes) -> cudaError_t {
    if (*ptr && bytes != old_bytes) {
      cudaFree(*ptr);
      *ptr = nullptr;
    }
    if (!*ptr) return cudaMalloc(ptr, bytes);
    return cudaSuccess;
  };
  if ((err = ensure(&G.tc_waves, sizeof(TCArgs) * W, sizeof(TCArgs) * W)) != cudaSuccess) return err;
  if ((err = ensure(reinterpret_cast<void**>(&G.maps), sizeof(CUtensorMap) * 3 * W, sizeof(CUtensorMap) * 3 * W)) !=
      cudaSuccess)
    return err;
  if ((err = ensure(&G.dslice_waves, sizeof(DSliceWave) * W, sizeof(DSliceWave) * W)) != cudaSuccess) return err;
  if ((err = ensure(reinterpret_cast<void**>(&G.tiles), sizeof(int4) * tiles.size(), sizeof(int4) * G.n_tiles)) !=
      cudaSuccess)
    return err;
  if ((err = ensure(&G.near_waves, sizeof(NearWave) * W, sizeof(NearWave) * W)) != cudaSuccess) return err;
  if ((err = ensure(reinterpret_cast<void**>(&G.near_jobs), sizeof(int2) * jobs.size(),
                    sizeof(int2) * G.n_near_jobs)) != cudaSuccess)
    return err;
  G.n_tiles = (int)tiles.size();
  if (G.n_tiles > 65535) G.tc_pair = false;  // the 2-SM launch holds the pair tiles in grid.y
  G.n_near_jobs = (int)jobs.size();
  if ((err = cudaMemcpy(G.tc_waves, tw.data(), sizeof(TCArgs) * W, cudaMemcpyHostToDevice)) != cudaSuccess) return err;
  if ((err = cudaMemcpy(G.maps, maps.data(), sizeof(CUtensorMap) * 3 * W, cudaMemcpyHostToDevice)) != cudaSuccess)
    return err;
  if ((err = cudaMemcpy(G.dslice_waves, dw.data(), sizeof(DSliceWave) * W, cudaMemcpyHostToDevice)) != cudaSuccess)
    return err;
  if ((err = cudaMemcpy(G.tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
    return err;
  if ((err = cudaMemcpy(G.near_waves, nw.data(), sizeof(NearWave) * W, cudaMemcpyHostToDevice)) != cudaSuccess)
    return err;
  if ((err = cudaMemcpy(G.near_jobs, jobs.data(), sizeof(int2) * jobs.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
    return err;
  if ((err = set_tc_smem()) != cudaSuccess) return err;
  return cudaFuncSetAttribute(near_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)near_smem_bytes(p.nR_max));
}

bool polesum_cluster_ok(int cx, int cy, int ns, bool pair) {
  GroupedFn fn = grouped_fn(cx, cy, cx == 1, ns, pair);
  if (!fn) return false;
  if (cx * cy == 1) return true;
  if (set_tc_smem() != cudaSuccess) return false;
  const bool two_sm = pair_applies(cx, cy, cx == 1, ns, pair);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = two_sm ? dim3(2, 8, 8) : dim3(cx * 8, cy * 8, 1);
  cfg.blockDim = dim3(two_sm ? PAIR_NTHREADS : NTHREADS, 1, 1);
  cfg.dynamicSmemBytes = grouped_smem(cx, cy, cx == 1, ns, pair);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = two_sm ? 2 : cx;
  attr[0].val.clusterDim.y = two_sm ? 1 : cy;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n > 0;
}

cudaError_t launch_polesum_split_grouped(const Plan& p, int64_t e0, int ne, cudaStream_t s) {
  if (ne <= 0) return cudaSuccess;
  const GroupDev& G = p.grp;
  const int ns = polesum_slice_planes(p.slices);
  GroupedFn fn = grouped_fn(G.tc_cx, G.tc_cy, G.dt(), ns, G.tc_pair);
  if (!fn) return cudaErrorInvalidValue;
  const int ny = (ne + BN - 1) / BN;
  const bool two_sm = pair_applies(G.tc_cx, G.tc_cy, G.dt(), ns, G.tc_pair);
  cudaLaunchConfig_t cfg = {};
  // the 2-SM kernel: grid (rank in pair, pair tile, energy-tile pair), clusters of 2 x 1 x 1
  cfg.gridDim = two_sm ? dim3(2, G.n_tiles, (ny + 1) / 2)
                       : dim3(G.n_tiles, (ny + G.tc_cy - 1) / G.tc_cy * G.tc_cy, 1);
  cfg.blockDim = dim3(two_sm ? PAIR_NTHREADS : NTHREADS, 1, 1);
  cfg.dynamicSmemBytes = grouped_smem(G.tc_cx, G.tc_cy, G.dt(), ns, G.tc_pair);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = two_sm ? 2 : G.tc_cx;
  attr[0].val.clusterDim.y = two_sm ? 1 : G.tc_cy;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = (G.tc_cx * G.tc_cy > 1) ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, fn, reinterpret_cast<const TCArgs*>(G.tc_waves), (const CUtensorMap*)G.maps,
                            (const int4*)G.tiles, e0, ne);
}

cudaError_t launch_near_grouped(const Plan& p, int64_t e0, int ne, cudaStream_t s) {
  if (ne <= 0) return cudaSuccess;
  const GroupDev& G = p.grp;
  dim3 grid(G.n_near_jobs, G.near_splits);
  near_grouped_kernel<<<grid, NNT, near_smem_bytes(p.nR_max), s>>>(reinterpret_cast<const NearWave*>(G.near_waves),
                                                                  G.near_jobs, e0, ne, G.near_splits);
  return cudaGetLastError();
}

cudaError_t launch_dslice_grouped(const Plan& p, int64_t e0, int ne, cudaStream_t s) {
  if (ne <= 0) return cudaSuccess;
  const GroupDev& G = p.grp;
  if (G.d_rows <= 0) return cudaErrorInvalidValue;
  // rows of the last 128-energy tile past ne are zeroed too (the MMAs read whole tiles)
  int rows = (ne + BN - 1) / BN * BN;
  if (rows > G.d_rows) rows = G.d_rows;
  dslice_grouped_kernel<<<dim3(rows, p.n_waves), 256, 0, s>>>(reinterpret_cast<const DSliceWave*>(G.dslice_waves), e0,
                                                               ne);
  return cudaGetLastError();
}

RM_CHECK_READER(polesum_tc)

}  // namespace rm
