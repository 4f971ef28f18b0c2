// BF16 / FP16 tensor-core fused GCDF kernel (tcgen05 + TMEM + TMA), sm_103a.
//
// What it computes per (waypoint i, point j) pair — the same network and
// reverse sweep as the FP32 path (Sec. III-C network, Sec. IV-A batched values
// and gradients):
//   z_1 = A_i + W_1p p_j,  h_l = s(z_l),  z_{l+1} = W_{l+1} h_l + b_{l+1},
//   f = w_o . s(z_L) + b_o,
//   g_L = w_o * s'(z_L),  g_{l-1} = (W_l^T g_l) * s'(z_{l-1}),  df/denc = W_1q^T g_1,
// followed by the sin/cos chain rule and either per-pair outputs or a
// per-tile partial of the min / soft-min / hinge reduction.
//
// Mapping onto the GPU.  CTAs run in clusters of two, one CTA per SM; each
// CTA owns a tile of 128 pairs of one waypoint and the pair's MMAs are 2-SM
// tcgen05 MMAs (cta_group::2, M = 256) issued by the even CTA: each CTA holds
// the A operand of its own 128 rows and half of every weight slab, so every
// SM receives half the weight bytes (weight streaming from L2 is what bounds a
// CTA that reloads the whole network for each tile).
//
// Two tiles in flight per CTA pair ("slots" 0 and 1).  Each H x H product of
// the forward pass or the reverse sweep ("a step") is one MMA chain of N = 256
// output columns, D (TMEM, FP32) = A (shared, 16-bit, 128 pairs x 256 per CTA)
// x B (shared, 16-bit weight rows, 128 per CTA), so a step reads its A operand
// once.  The tensor core alternates between the slots: while it computes a step
// of one slot, the epilogue turns the other slot's last step into that slot's
// next operand, so neither waits for the other as long as an epilogue step is
// shorter than a step of MMAs.  Each slot has one A buffer (its step's
// epilogue writes the next operand into it once the step's MMAs have read it)
// and one 256-column accumulator.  Weights stream through a ring of 16 KB
// stages (one K = 64 slab: each CTA's 128 weight rows as two 64-row boxes)
// loaded by TMA in the order the MMAs consume them; both CTAs' loads of a stage
// complete on one barrier of the even CTA, and the even CTA's commit releases
// the stage in both.  The reverse operands are stored copies of W_l^T scaled
// by 1/2 (exact), so both directions are K-major.
//
// Epilogue arithmetic (packed FP16 pairs):
//   u = z / 2 = acc / 2 + b / 2,  t = tanh(u),  s(z) = z sigma(z) = u (1 + t),
//   2 s'(z) = (1 + t) + s(z) (1 - t)
// (BF16 operands: s(z) = u (1 + t) formed exactly in FP32 and rounded once).
// 2 s'(z_l) of layers 1..L-1 goes to a per-CTA stash in global memory as FP16
// pairs ([slot][layer][8-column chunk][row], 16 bytes: each warp store or load
// covers 512 contiguous bytes; 128 KB per CTA and layer, so it stays in L2),
// written by the epilogue that computes s(z_l) (the first layer's by the tile's
// first-layer pass) and read back by the reverse step that needs it; the
// halved reverse operands cancel the factor 2.  The output sum
// f = w_o . s(z_L) accumulates in FP32.
//
// TMEM columns (512, allocated for the CTA pair): slot s's accumulator is
// [256 s, 256 s + 256), columns [0, 128) ("half a") first; the input-Jacobian
// chain (N = 32) of a slot writes the first 32 columns of its half b after the
// last reverse step has been read.
//
// Tile boundary: the slot's next tile's inputs are fetched after its last
// reverse step; the tail reads the Jacobian and writes the next tile's first
// layer into the slot's A buffer before its output stage (chain rule,
// reduction), so the slot's next chain can start early; slot 0 runs one item
// ahead of slot 1.
//
// Warp roles (608 threads per CTA): warp 0 issues TMA loads, warp 1 allocates
// TMEM and (even CTA) issues the pair's MMAs, warp 18 merges each tile's four
// row-quad partial records into the tile's record, warps 2..17 are the
// epilogue: thread = one pair row (TMEM lane) and 64 columns; the 8 warps of
// columns [0, 128) and the 8 of [128, 256) each signal their half to the MMA
// issuer with one arrival per warp; the next chain starts once both halves of
// both CTAs have arrived (its first MMA overwrites the whole accumulator).
// The input-Jacobian operand W_1q^T streams through the same ring as the
// weights.
//
// Every cross-warp and cross-CTA handoff is an mbarrier and every wait on one
// is bounded (about a second).  On expiry the kernel records an error in a
// device status word, stops issuing work, drains its outstanding copies and
// MMAs and frees TMEM before returning; both CTAs of a pair always reach the
// closing cluster barrier.
#include <cstring>
#include <vector>

#include "gcdf_internal.cuh"
#include "tc_ptx.cuh"

namespace gcdf {

namespace {

constexpr int kTile = 128;             // pairs per CTA tile; a CTA pair shares each MMA (M = 256)
constexpr int kH = 256;                // hidden width handled by this kernel
constexpr int kHalf = 128;             // accumulator columns per half (one CTA's share of a step's weight rows)
constexpr int kRowsCta = kHalf / 2;    // weight rows per TMA box (two boxes per CTA and stage)
constexpr int kSlots = 2;              // tiles in flight per CTA pair
constexpr int kStages = 4;             // weight ring depth
constexpr int kSlabBytes = kRowsCta * 128;  // 64 rows x 64 16-bit values (one K = 64 slab)
constexpr int kStageBytes = 2 * kSlabBytes; // one stage: 16 KB per CTA
constexpr int kABytes = kTile * kH * 2;
constexpr int kThreads = 608;          // 19 warps
constexpr int kMergeWarp = 18;         // merges each tile's four row-quad records
constexpr int kEpiThreads = 512;       // epilogue threads (16 warps)
constexpr int kEpiWarps = 16;
constexpr uint32_t kTmemCols = 512;    // one 256-column FP32 accumulator per slot

// shared memory map (offsets from the 1024-aligned base)
constexpr int kOffA0 = 0;                                       // slot 0's operand buffer
constexpr int kOffA1 = kABytes;                                 // slot 1's
constexpr int kOffRing = 2 * kABytes;                           // 131072
constexpr int kOffBiasH = kOffRing + kStages * kStageBytes;      // [(L-1) x H/2] f16x2 b_l / 2, L <= 4
constexpr int kOffW1p = kOffBiasH + 3 * (kH / 2) * 4;           // [H/2] uint4: f16x2 W_1p / 2 (x, y, z pairs)
constexpr int kOffWo = kOffW1p + (kH / 2) * 16;                 // [H] fp32 w_o
constexpr int kOffWoh = kOffWo + kH * 4;                        // [H/2] f16x2 w_o / 2
constexpr int kOffAiw = kOffWoh + (kH / 2) * 4;                 // [2 slots][16 warps][32] f16x2 A_i / 2
constexpr int kOffPt = kOffAiw + kSlots * kEpiWarps * 32 * 4;   // [2 slots][128 rows] uint4: the row's point, packed
constexpr int kOffTrig = kOffPt + kSlots * kTile * 16;          // [2 slots][2 tiles][16 warps][24] sin, cos
constexpr int kOffTinfo = kOffTrig + kSlots * 2 * kEpiWarps * 24 * 4;  // [2 slots][2 tiles][16 warps] int4 tile
constexpr int kOffF = kOffTinfo + kSlots * 2 * kEpiWarps * 16;  // [2 slots][2 tiles][4][128] f partials
constexpr int kOffPart = kOffF + kSlots * 2 * 4 * kTile * 4;    // 4 partial records
constexpr int kOffBar = kOffPart + 4 * (int)sizeof(Partial);
constexpr int kNumBars = 2 * kStages + 16;
constexpr int kOffSlot = kOffBar + kNumBars * 8;
constexpr int kSmemBytes = kOffSlot + 16 + 1024;                // + alignment slack
static_assert(kSmemBytes <= 227 * 1024 - 64, "shared memory budget");
static_assert(kOffPt % 16 == 0 && kOffTinfo % 16 == 0 && kOffBar % 8 == 0, "alignment");

// barrier indices
constexpr int B_FULL0 = 0;              // + stage: both CTAs' slabs landed (used in the even CTA)
constexpr int B_EMPTY0 = kStages;       // + stage: its MMAs completed (commit to both CTAs)
constexpr int B_ACC0 = 2 * kStages;     // + slot: the slot's step complete (commit to both CTAs)
constexpr int B_ACCJ0 = 2 * kStages + 2;  // + slot: input-Jacobian chain complete (commit to both CTAs)
constexpr int B_FD0 = 2 * kStages + 4;  // + slot: f partials written (512 arrivals)
constexpr int B_ED0 = 2 * kStages + 6;  // + 2 slot + half: epilogues of both CTAs done (even CTA, 16 warp arrivals)
// + 2 slot + half: a tile's first layer written (even CTA, 16 warp arrivals).
// Kept apart from B_ED0: a warp arrives for its last reverse step and later for
// the next tile's first layer; on one barrier a fast warp's second arrival could
// complete the phase that still waits for a slow warp's first.
constexpr int B_FL0 = 2 * kStages + 10;
constexpr int B_PD = 2 * kStages + 14;  // partial-record parts written (16 warp arrivals)
constexpr int B_MD = 2 * kStages + 15;  // the merge warp has read them (1 arrival)

constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at GB300 clocks

__device__ __forceinline__ uint32_t bar(uint32_t base, int i) { return base + kOffBar + 8 * i; }

// Wait used by the single-thread producer and MMA roles: gives up early when
// another role has aborted.  `limit` (cycles) is kWaitCycles except in the
// expiry self-test.
__device__ __forceinline__ bool wait_role(uint32_t b, uint32_t parity, volatile int* abort_flag, int* err,
                                          long long limit = kWaitCycles) {
  if (ptx::mbar_try_wait(b, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (ptx::mbar_try_wait(b, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > limit) {
      *abort_flag = 1;
      atomicOr(err, 1);
      return false;
    }
  }
}

// Wait used by epilogue threads: only its own time limit ends it, so every
// thread waiting on the same phase takes the same decision.  Waiting threads
// sleep in hardware rather than poll, leaving issue slots to working warps.
__device__ __forceinline__ bool wait_epi(uint32_t b, uint32_t parity, volatile int* abort_flag, int* err,
                                         long long limit = kWaitCycles) {
  if (ptx::mbar_try_wait(b, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (ptx::mbar_try_wait_sleep(b, parity, 100000u)) return true;
    if (clock64() - t0 > limit) {
      *abort_flag = 1;
      atomicOr(err, 1);
      return false;
    }
  }
}

// wait_epi by every lane of a warp, with one decision for the whole warp (the
// epilogue synchronises its warps, so no lane may leave a loop alone)
__device__ __forceinline__ bool wait_epi_warp(uint32_t b, uint32_t parity, volatile int* abort_flag, int* err,
                                              long long limit = kWaitCycles) {
  const bool got = wait_epi(b, parity, abort_flag, err, limit);
  return __all_sync(0xffffffffu, got);
}

// Self-test of the bounded waits (gcdf_selftest_wait_expiry): one CTA of two
// warps waits, with the fused kernel's own helpers, on an mbarrier that nothing
// ever arrives on.  Warp 0's lane 0 takes the producer / MMA wait, warp 1 the
// epilogue's warp-wide wait; both must give up after `limit` cycles, raise the
// abort flag and set bit 0 of the status word.  No copy, MMA or tensor memory
// is involved, so nothing is left in flight when the waits expire.
// seen[0] / seen[1]: 1 when the producer / epilogue wait returned "expired",
// seen[2]: the abort flag afterwards.
__global__ void __launch_bounds__(64, 1) wait_expiry_probe_kernel(int* err, long long limit, int* seen) {
  __shared__ __align__(8) uint64_t never;
  __shared__ int abort_flag_s;
  volatile int* abort_flag = &abort_flag_s;
  const uint32_t b = ptx::smem_u32(&never);
  if (threadIdx.x == 0) {
    abort_flag_s = 0;
    ptx::mbar_init(b, 1);
    ptx::fence_barrier_init();
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    if (lane == 0) {
      // gives up at its own limit or when the other warp's expiry raised the flag
      const bool got = wait_role(b, 0u, abort_flag, err, limit);
      seen[0] = got ? 0 : 1;
    }
  } else {
    const bool got = wait_epi_warp(b, 0u, abort_flag, err, limit);
    if (lane == 0) seen[1] = got ? 0 : 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) seen[2] = abort_flag_s;
}

__device__ __forceinline__ int total_tiles(const WorkDesc& w) {
  return w.tile_start ? w.tile_start[w.N] : w.n_tiles;
}

constexpr uint32_t kOne2 = 0x3C003C00u;   // (1.0, 1.0) in FP16
constexpr uint32_t kHalf2 = 0x38003800u;  // (0.5, 0.5) in FP16
constexpr float kGradScale8 = 64.f;         // FP8 reverse operands hold 64 g (E4M3 normals start at 2^-6)

// Packed SiLU of u = z / 2: returns s(z) and 2 s'(z) for two values.
__device__ __forceinline__ void silu2(uint32_t u, uint32_t& h, uint32_t& s2) {
  const uint32_t t = ptx::htanh2(u);
  h = ptx::hfma2(u, t, u);
  s2 = ptx::hfma2(h, ptx::hsub2(kOne2, t), ptx::hadd2(kOne2, t));
}

// The same for the BF16 operand path: s(z) = u (1 + t) is formed exactly in
// FP32 from the FP16 factors and rounded once to BF16 (no FP16 rounding of s(z)
// and no FP16 -> BF16 conversion); 2 s'(z) = (1 + t) + (1 + t)(u - u t).
__device__ __forceinline__ void silu2_bf16(uint32_t u, uint32_t& h_bf16, uint32_t& s2) {
  const uint32_t t = ptx::htanh2(u);
  const uint32_t tp1 = ptx::hadd2(kOne2, t);
  float h0, h1;
  ptx::f16x2_products(u, tp1, h0, h1);
  h_bf16 = ptx::pack_bf16x2(h0, h1);
  s2 = ptx::hfma2(tp1, ptx::hfnms2(u, t), tp1);
}

template <int kFmt>
__device__ __forceinline__ uint32_t to_operand(uint32_t f16pair) {
  // BF16 converts here; FP16 is the operand; FP8 is converted where it is stored
  return kFmt == 0 ? ptx::f16x2_to_bf16x2(f16pair) : f16pair;
}

// u_1 = z_1 / 2 for columns c, c+1 of this thread's pair in packed FP16:
// A_i / 2 + (W_1p / 2) p, one fused multiply-add per point coordinate.
__device__ __forceinline__ uint32_t first_layer_u2(uint4 w, uint32_t ah, uint32_t px2, uint32_t py2, uint32_t pz2) {
  return ptx::hfma2(w.z, pz2, ptx::hfma2(w.y, py2, ptx::hfma2(w.x, px2, ah)));
}

// Minimum over the 32 lanes of a warp (no NaN among the inputs).
__device__ __forceinline__ float warp_min(float x) {
  float r;
  asm volatile("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(x));
  return r;
}

// Part of the per-tile partial record of a row quad: the 32 rows of a warp (lane =
// row; the list position grows with the lane) reduced for the gradient components
// d = d0, d0 + 4, d0 + 8 held in dqm[] (zero past n).  The four warps of the quad
// (d0 = 0..3) compute the same argmin and weights and write disjoint fields of
// *out; the warp with d0 = 0 also writes the value fields and the argmin.
// Argmin by (f, list position) with NaN first: a NaN ballot, else the warp minimum
// (redux) and the lowest lane holding it.  SOFTMIN takes one exponential per row
// relative to the warp minimum.  Sums use a fixed butterfly (deterministic).
__device__ __forceinline__ void warp_partial_part(int mode, float param, bool valid, float f, const float* dqm,
                                                  int d0, int n, int idx, int pos, Partial* out) {
  const int lane = threadIdx.x & 31;
  float* rec = reinterpret_cast<float*>(out);  // v0, v1, idx, pos, g[kMaxDof]
  const unsigned nanm = __ballot_sync(0xffffffffu, valid && f != f);
  float fm;
  unsigned win;
  if (nanm) {
    win = nanm;
    fm = __int_as_float(0x7fc00000);
  } else {
    const float fv = valid ? f : __int_as_float(0x7f800000);
    fm = warp_min(fv);
    win = __ballot_sync(0xffffffffu, valid && fv == fm);
  }
  if (win == 0u) {  // no valid row
    if (d0 == 0 && lane == 0) *out = partial_identity(mode);
    return;
  }
  const int src = __ffs(win) - 1;
  if (mode == kMin) {
    if (lane == src) {
      if (d0 == 0) {
        rec[0] = f;
        rec[1] = 0.f;
        reinterpret_cast<int*>(rec)[2] = idx;
        reinterpret_cast<int*>(rec)[3] = pos;
      }
#pragma unroll
      for (int m = 0; m < 3; ++m) rec[4 + d0 + 4 * m] = dqm[m];
    }
    return;
  }
  float wgt, v0;
  if (mode == kSoftmin) {
    wgt = valid ? __expf(-(f - fm) / param) : 0.f;
    if (valid && f != f) wgt = f;
    v0 = 0.f;
  } else {
    wgt = (valid && f < param) ? -1.f : 0.f;
    v0 = valid ? fmaxf(0.f, param - f) : 0.f;
    if (valid && f != f) v0 = f;
  }
  float v[4];
  // HINGE selects the active rows' gradients (an inactive row adds nothing,
  // not 0 x its gradient: a NaN or infinite gradient of an inactive row must
  // not reach the sum)
#pragma unroll
  for (int m = 0; m < 3; ++m) v[m] = (d0 + 4 * m < n && (mode == kSoftmin || wgt != 0.f)) ? wgt * dqm[m] : 0.f;
  v[3] = (mode == kSoftmin) ? wgt : v0;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1)
#pragma unroll
    for (int m = 0; m < 4; ++m) v[m] += __shfl_xor_sync(0xffffffffu, v[m], o);
  if (lane == 0) {
#pragma unroll
    for (int m = 0; m < 3; ++m) rec[4 + d0 + 4 * m] = v[m];
    if (d0 == 0) rec[mode == kSoftmin ? 1 : 0] = v[3];
  }
  if (d0 == 0 && lane == src) {
    rec[mode == kSoftmin ? 0 : 1] = fm;
    reinterpret_cast<int*>(rec)[2] = idx;
    reinterpret_cast<int*>(rec)[3] = pos;
  }
}

// Merge of the four row-quad records of a tile into rec_out (global), one field
// per lane (lanes 0..15), the result of folding them left to right with
// partial_combine up to rounding: winner by (min f, position) with NaN first;
// SOFTMIN rescales every record to the winner's minimum (one exponential per
// record), HINGE adds the hinge sums.
__device__ __forceinline__ void warp_combine_quads(int mode, float T, const Partial* parts, Partial* rec_out) {
  const int lane = threadIdx.x & 31;
  const float* R = reinterpret_cast<const float*>(parts);
  const int* Ri = reinterpret_cast<const int*>(parts);
  constexpr int kF = (int)(sizeof(Partial) / 4);
  int wq = -1;
  float wf = 0.f;
  int wp = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int pq = Ri[q * kF + 3];
    if (pq == 0x7fffffff) continue;  // identity record
    const float fq = (mode == kHinge) ? R[q * kF + 1] : R[q * kF + 0];
    if (wq < 0 || first_is_better(fq, pq, wf, wp)) {
      wq = q;
      wf = fq;
      wp = pq;
    }
  }
  float eq = 1.f;  // SOFTMIN rescale factor of record `lane` (lanes 0..3)
  if (mode == kSoftmin && wq >= 0 && lane < 4) {
    const float m = R[wq * kF + 0], v0 = R[lane * kF + 0];
    eq = (v0 == m) ? 1.f : __expf(-(v0 - m) / T);
  }
  float e4[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) e4[q] = __shfl_sync(0xffffffffu, eq, q);
  if (lane >= kF) return;
  float* out = reinterpret_cast<float*>(rec_out);
  if (wq < 0) {  // the identity record, field by field (as partial_identity)
    float v = 0.f;
    if (lane == 0) v = (mode == kHinge) ? 0.f : __int_as_float(0x7f800000);
    if (lane == 1) v = (mode == kHinge) ? __int_as_float(0x7f800000) : 0.f;
    if (lane == 2) v = __int_as_float(-1);
    if (lane == 3) v = __int_as_float(0x7fffffff);
    out[lane] = v;
    return;
  }
  if (mode == kMin || lane == 2 || lane == 3) {
    out[lane] = R[wq * kF + lane];
    return;
  }
  if (mode == kHinge && lane == 1) {
    out[1] = R[wq * kF + 1];
    return;
  }
  if (mode == kSoftmin && lane == 0) {
    out[0] = R[wq * kF + 0];
    return;
  }
  float acc = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (Ri[q * kF + 3] != 0x7fffffff) acc += R[q * kF + lane] * e4[q];
  out[lane] = acc;
}

// The order in which every role of a CTA pair (TMA producer, MMA issuer,
// epilogue, merge warp) takes its work items.  Slot 0 holds the cluster's even
// local tiles, slot 1 the odd ones; a tile is n_items items (its weight steps,
// then its tail: the input-Jacobian chain and output stage).  Slot 0 runs
// `lead` items alone, then the two slots alternate, so that while the tensor
// core computes one slot's step the epilogue turns the other slot's previous
// step into its next operand.  (A lead of one item measured 0.5 % faster in
// BF16 and 1.7 % in FP16 than three or five, which put the two slots' tile
// boundaries further apart.)
struct Schedule {
  int n_items, ni0, ni1, k0, k1, lead;
  __device__ __forceinline__ bool next(int& slot, int& tile_local, int& step) {
    const bool have0 = k0 < ni0, have1 = k1 < ni1;
    if (!have0 && !have1) return false;
    const bool one = !have0 || (have1 && k0 >= lead && k1 <= k0 - lead);
    const int kk = one ? k1 : k0;
    if (one) ++k1; else ++k0;
    slot = one ? 1 : 0;
    tile_local = kk / n_items;
    step = kk - tile_local * n_items;
    return true;
  }
};

// kFmt: operand format, 0 = BF16, 1 = FP16, 2 = FP8 E4M3 (per-layer scales).
// kFwd: value-only queries (the forward steps alone), a separate instantiation
// so that the full sweep carries none of its branches.
template <int kFmt, bool kFwd>
__global__ void __launch_bounds__(kThreads, 1)
tc_fused_kernel(const WorkDesc w, const __grid_constant__ CUtensorMap map_w,
                const __grid_constant__ CUtensorMap map_j, const TcWeights tw) {
  constexpr bool kF16 = kFmt == 1;
  constexpr bool kF8 = kFmt == 2;
  // A 128-byte slab row holds K = 64 16-bit or K = 128 FP8 values; a weight
  // step (N = 256, K = 256) takes 4 or 2 ring stages of one slab each.  An
  // input-Jacobian stage (N = 32) holds K = 128: two 16-bit slabs or one FP8 slab.
  constexpr int kSlabK = kF8 ? 128 : 64;
  constexpr int kStagesPerStep = kH / kSlabK;
  constexpr int kSlabsPerStage = kF8 ? 1 : 2;  // input-Jacobian stages
  extern __shared__ uint8_t smem_raw[];
  const uint32_t base = (ptx::smem_u32(smem_raw) + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - ptx::smem_u32(smem_raw));
  __shared__ int abort_flag_s;
  volatile int* abort_flag = &abort_flag_s;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int L = tw.L;
  // A query without a gradient output (value-only) runs the forward steps
  // alone: no stash, no reverse steps, no input-Jacobian chain.
  constexpr bool fwd = kFwd;  // launched for w.mode == kQuery with w.g_out == nullptr
  const int n_steps = fwd ? (L - 1) : 2 * (L - 1);  // weight steps per tile (forward, then reverse)
  const int nj = tw.nj;
  const int ntiles = total_tiles(w);
  // CTA pairs (clusters of 2) take pair tiles round robin; CTA `rank` of the pair
  // owns tile 2 k + rank of pair tile k (past the last tile: an empty tile)
  const uint32_t rank = ptx::cluster_ctarank();
  const bool leader = (rank == 0);
  const int cluster = (int)blockIdx.x >> 1;
  const int nclusters = (int)gridDim.x >> 1;
  const int npt = (ntiles + 1) >> 1;
  int my_tiles = 0;  // pair tiles of this cluster (the same for both CTAs)
  if (cluster < npt) my_tiles = (npt - 1 - cluster) / nclusters + 1;

  uint32_t* s_biasH = reinterpret_cast<uint32_t*>(gbase + kOffBiasH);
  uint4* s_w1p = reinterpret_cast<uint4*>(gbase + kOffW1p);
  float* s_wo = reinterpret_cast<float*>(gbase + kOffWo);
  uint32_t* s_woh = reinterpret_cast<uint32_t*>(gbase + kOffWoh);
  float* s_f = reinterpret_cast<float*>(gbase + kOffF);
  Partial* s_part = reinterpret_cast<Partial*>(gbase + kOffPart);
  uint32_t* s_slot = reinterpret_cast<uint32_t*>(gbase + kOffSlot);

  // ---- setup -------------------------------------------------------------------
  if (tid == 0) {
    abort_flag_s = 0;
    for (int s = 0; s < kStages; ++s) {
      ptx::mbar_init(bar(base, B_FULL0 + s), 1);
      ptx::mbar_init(bar(base, B_EMPTY0 + s), 1);
    }
    for (int sl = 0; sl < kSlots; ++sl) {
      ptx::mbar_init(bar(base, B_ACC0 + sl), 1);
      ptx::mbar_init(bar(base, B_ACCJ0 + sl), 1);
      ptx::mbar_init(bar(base, B_FD0 + sl), kEpiThreads);
      for (int h = 0; h < 2; ++h) {
        ptx::mbar_init(bar(base, B_ED0 + 2 * sl + h), kEpiWarps);  // 8 warps of the half x 2 CTAs
        ptx::mbar_init(bar(base, B_FL0 + 2 * sl + h), kEpiWarps);
      }
    }
    ptx::mbar_init(bar(base, B_PD), kEpiWarps);
    ptx::mbar_init(bar(base, B_MD), 1);
    ptx::fence_barrier_init();
    ptx::prefetch_tensormap(&map_w);
    ptx::prefetch_tensormap(&map_j);
  }
  if (warp == 1) {
    ptx::tmem_alloc_pair(base + kOffSlot, kTmemCols);
    ptx::tmem_relinquish_pair();
  }
  for (int c = tid; c < kH; c += kThreads) s_wo[c] = tw.wout[c];
  for (int i = tid; i < kH / 2; i += kThreads) {
    const int c = 2 * i;
    s_w1p[i] = make_uint4(ptx::pack_f16x2(0.5f * tw.W1p[3 * c], 0.5f * tw.W1p[3 * c + 3]),
                          ptx::pack_f16x2(0.5f * tw.W1p[3 * c + 1], 0.5f * tw.W1p[3 * c + 4]),
                          ptx::pack_f16x2(0.5f * tw.W1p[3 * c + 2], 0.5f * tw.W1p[3 * c + 5]), 0u);
    const float gs = kF8 ? 0.5f * kGradScale8 : 0.5f;  // FP8 gradient operands carry x64
    s_woh[i] = ptx::pack_f16x2(gs * tw.wout[c], gs * tw.wout[c + 1]);
  }
  for (int i = tid; i < (L - 1) * (kH / 2); i += kThreads) {
    const int l = i / (kH / 2), c = 2 * (i % (kH / 2));
    s_biasH[i] = ptx::pack_f16x2(0.5f * tw.bias[(size_t)l * kH + c], 0.5f * tw.bias[(size_t)l * kH + c + 1]);
  }
  // both CTAs' barriers are initialised before either signals the other's
  ptx::tc_fence_before();
  ptx::cluster_sync();
  ptx::tc_fence_after();
  const uint32_t tmem = *s_slot;

  // Every role walks the same sequence of work items (Schedule): slot 0 takes
  // the cluster's even local tiles, slot 1 the odd ones; a tile is n_steps
  // weight steps and one tail item.
  const int n_items = n_steps + 1;
  auto make_sched = [&]() {
    Schedule sc;
    sc.n_items = n_items;
    sc.ni0 = ((my_tiles + 1) >> 1) * n_items;
    sc.ni1 = (my_tiles >> 1) * n_items;
    sc.k0 = sc.k1 = 0;
    sc.lead = 1;
    return sc;
  };

  if (warp == 0) {
    // ================= TMA producer (both CTAs) =================
    // A step's stage holds one 128-byte-wide K slab (K = 64 of 16-bit operands,
    // K = 128 of FP8) of this CTA's 128 weight rows (the step's N = 256 output
    // rows are split between the two CTAs), loaded as two 64-row boxes; an
    // input-Jacobian stage holds K = 128 of its nj / 2 rows.  Both CTAs' loads
    // complete on the even CTA's FULL barrier; each CTA refills a stage once the
    // MMAs that read it have completed (the even CTA's commit arrives on both
    // CTAs' EMPTY barriers).
    if (lane == 0 && my_tiles > 0) {
      const uint32_t full_lead = ptx::mapa_shared(bar(base, B_FULL0), 0);
      long long g = 0;         // stages issued
      int pst = 0;             // ring stage of g
      uint32_t puse = 0;       // (g / kStages) & 1
      bool ok = true;
      // dx, dy: offset of the second box (the next K slab of the same rows, or
      // the next 64 rows of the same K slab); none for FP8 Jacobian stages
      auto load_stage = [&](const CUtensorMap* map, int x0, int y, int dx, int dy, bool two,
                            uint32_t box_bytes) -> bool {
        const int st = pst;
        if (g >= kStages && !wait_role(bar(base, B_EMPTY0 + st), puse ^ 1u, abort_flag, tw.err)) return false;
        const uint32_t fb = full_lead + 8u * (uint32_t)st;
        // boxes x 2 CTAs
        if (leader) ptx::mbar_arrive_expect_tx(bar(base, B_FULL0 + st), 2u * (two ? 2u : 1u) * box_bytes);
        ptx::tma_load_2d_pair(base + kOffRing + st * kStageBytes, map, x0, y, fb);
        if (two) ptx::tma_load_2d_pair(base + kOffRing + st * kStageBytes + kSlabBytes, map, x0 + dx, y + dy, fb);
        ++g;
        if (++pst == kStages) { pst = 0; puse ^= 1u; }
        return true;
      };
      Schedule sc = make_sched();
      int slot, jl, s;
      while (ok && sc.next(slot, jl, s)) {
        if (s < n_steps) {
          const int row0 = (s < L - 1) ? s * kH : (L - 1 + (2 * L - 3 - s)) * kH;
          for (int k = 0; k < kStagesPerStep && ok; ++k)
            ok = load_stage(&map_w, k * kSlabK, row0 + (int)rank * kHalf, 0, kRowsCta, true, kSlabBytes);
        } else if (!fwd) {  // W_1q^T: nj rows, nj / 2 per CTA
          for (int pr = 0; pr < 2 && ok; ++pr)
            ok = load_stage(&map_j, pr * 128, (int)rank * (nj / 2), 64, 0, !kF8, (uint32_t)(nj / 2) * 128u);
        }
      }
      // drain (even CTA): the last kStages stages are the only ones that can be
      // in flight; their FULL phases cover both CTAs' loads
      if (leader) {
        for (long long k = (g > kStages ? g - kStages : 0); k < g; ++k) {
          const long long t0 = clock64();
          while (!ptx::mbar_try_wait(bar(base, B_FULL0 + (int)(k % kStages)), (uint32_t)(k / kStages) & 1u))
            if (clock64() - t0 > kWaitCycles) { atomicOr(tw.err, 2); break; }
        }
      }
    }
  } else if (warp == 1) {
    // ================= MMA issuer (even CTA, for both) =================
    if (lane == 0 && my_tiles > 0 && leader) {
      // (E4M3 x E4M3 has the format code 0 of FP16 x FP16 in the same fields)
      const uint32_t id256 = ptx::idesc_f16kind(2 * kTile, kH, kF16 || kF8);
      const uint32_t idj = ptx::idesc_f16kind(2 * kTile, nj, kF16 || kF8);
      long long g = 0;         // stages consumed
      int cst = 0;             // ring stage of g
      uint32_t cph = 0;        // its FULL phase parity
      // ED completions consumed per slot and half (scalars: a runtime-indexed
      // array would live in local memory)
      uint32_t ed00 = 0, ed01 = 0, ed10 = 0, ed11 = 0;
      bool ok = true;
      // Shared-memory descriptors are linear in the start address (bits 0-13 hold
      // address / 16), so every operand descriptor is a base plus a small offset;
      // the same offsets address the peer CTA's operands.
      // (selected, never indexed: a dynamically indexed array would live in local memory)
      const uint64_t dA0 = ptx::smem_desc_sw128(base + kOffA0, 1024), dA1 = ptx::smem_desc_sw128(base + kOffA1, 1024);
      const uint64_t dRing = ptx::smem_desc_sw128(base + kOffRing, 1024);
      // one weight-step stage: one K slab, 4 MMAs of N = 256 (32 bytes of K each),
      // then release the stage in both CTAs
      auto stage_mmas_w = [&](uint32_t dtm, uint64_t da, bool first) {
        const uint64_t db = dRing + (uint64_t)(cst * (kStageBytes >> 4));
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          if constexpr (kF8)
            ptx::mma_pair_f8(dtm, da + (uint64_t)(2 * ks), db + (uint64_t)(2 * ks), id256, (first && ks == 0) ? 0u : 1u);
          else
            ptx::mma_pair(dtm, da + (uint64_t)(2 * ks), db + (uint64_t)(2 * ks), id256, (first && ks == 0) ? 0u : 1u);
        }
        ptx::mma_commit_pair(bar(base, B_EMPTY0 + cst));
        ++g;
        if (++cst == kStages) { cst = 0; cph ^= 1u; }
      };
      // one input-Jacobian stage: K = 128 (8 MMAs of K = 16, or 4 of FP8 K = 32)
      auto stage_mmas = [&](uint32_t dtm, uint64_t da, uint32_t idd, bool first) {
        const uint64_t db = dRing + (uint64_t)(cst * (kStageBytes >> 4));
        // 32 bytes of K per MMA: K = 16 of 16-bit operands over two slabs, K = 32 of FP8 over one
        if constexpr (kF8) {
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)
            ptx::mma_pair_f8(dtm, da + (uint64_t)(2 * ks), db + (uint64_t)(2 * ks), idd, (first && ks == 0) ? 0u : 1u);
        } else {
#pragma unroll
          for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
              ptx::mma_pair(dtm, da + (uint64_t)(q * (kTile * 128 >> 4) + 2 * ks),
                            db + (uint64_t)(q * (kSlabBytes >> 4) + 2 * ks), idd, (first && q == 0 && ks == 0) ? 0u : 1u);
        }
        ptx::mma_commit_pair(bar(base, B_EMPTY0 + cst));
        ++g;
        if (++cst == kStages) { cst = 0; cph ^= 1u; }
      };
      Schedule sc = make_sched();
      int slot, jl, s;
      while (ok && sc.next(slot, jl, s)) {
        const bool jstep = (s == n_steps);
        if (fwd && jstep) continue;  // forward-only tiles have no MMA in their tail
        const uint64_t dAbuf = slot ? dA1 : dA0;
        // The operand's columns [128 h, 128 h + 128) come from the slot's previous
        // step's half h (both CTAs' epilogues arrive); step 0: the tile's first
        // layer, on its own barriers.  Either also proves that the warps of that
        // half have read their columns of the slot's accumulator (or, at step 0,
        // the Jacobian columns).  Every chain waits for both halves before its
        // first MMA: a step's first MMA writes the whole accumulator, and the
        // Jacobian chain writes columns of half b.
        auto wait_half = [&](int h) -> bool {
          const int bi = 2 * slot + h;
          const uint32_t edn = slot ? (h ? ed11 : ed10) : (h ? ed01 : ed00);
          const bool ok_w = (s == 0) ? wait_role(bar(base, B_FL0 + bi), (uint32_t)jl & 1u, abort_flag, tw.err)
                                     : wait_role(bar(base, B_ED0 + bi), edn & 1u, abort_flag, tw.err);
          if (ok_w && s != 0) {
            if (slot) { if (h) ++ed11; else ++ed10; }
            else { if (h) ++ed01; else ++ed00; }
          }
          ptx::tc_fence_after();
          return ok_w;
        };
        if (jstep) {
          // the input Jacobian df/denc = W_1q^T g_1 goes to the first nj columns of
          // the slot's accumulator half b (every warp reads it before it writes its
          // part of the next tile's first layer)
          const uint32_t dtm = tmem + (uint32_t)(slot * kH + kHalf);
          ok = wait_half(0) && wait_half(1);
#pragma unroll
          for (int pr = 0; pr < 2 && ok; ++pr) {
            if (!wait_role(bar(base, B_FULL0 + cst), cph, abort_flag, tw.err)) { ok = false; break; }
            stage_mmas(dtm, dAbuf + (uint64_t)((kSlabsPerStage * pr) * (kTile * 128) >> 4), idj, pr == 0);
          }
        } else {
          // one chain of N = 256 into the slot's accumulator: its A operand is read
          // once per step
          const uint32_t dtm = tmem + (uint32_t)(slot * kH);
          ok = wait_half(0) && wait_half(1);
#pragma unroll
          for (int k = 0; k < kStagesPerStep && ok; ++k) {
            if (!wait_role(bar(base, B_FULL0 + cst), cph, abort_flag, tw.err)) { ok = false; break; }
            stage_mmas_w(dtm, dAbuf + (uint64_t)(k * (kTile * 128 >> 4)), k == 0);
          }
        }
        // one commit per step: it tracks every earlier MMA of this thread, so the
        // chain (and with it every read of the slot's A buffer) is done
        if (ok) ptx::mma_commit_pair(bar(base, jstep ? B_ACCJ0 + slot : B_ACC0 + slot));
      }
      // all issued MMAs complete before TMEM is released: wait for the last
      // EMPTY arrivals (they follow every earlier MMA of this thread)
      for (long long k = (g > kStages ? g - kStages : 0); k < g; ++k) {
        const long long t0 = clock64();
        while (!ptx::mbar_try_wait(bar(base, B_EMPTY0 + (int)(k % kStages)), (uint32_t)(k / kStages) & 1u))
          if (clock64() - t0 > kWaitCycles) { atomicOr(tw.err, 2); break; }
      }
    }
  } else if (warp == kMergeWarp) {
    // ================= merge warp: one partial record per tile =================
    if (w.mode != kQuery) {
      Schedule sc = make_sched();
      int slot, jl, s;
      uint32_t n_out = 0;
      while (sc.next(slot, jl, s)) {
        if (s != n_steps) continue;
        if (!wait_epi_warp(bar(base, B_PD), n_out & 1u, abort_flag, tw.err)) break;
        const int it = 2 * jl + slot;
        const int t = 2 * (cluster + it * nclusters) + (int)rank;
        if (t < ntiles) warp_combine_quads(w.mode, w.param, s_part, &w.partials[t]);
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(bar(base, B_MD));  // s_part may be rewritten
        ++n_out;
      }
    }
  } else {
    // ================= epilogue: 16 warps, one pair row, 64 columns each ========
    const int e = warp - 2;
    const int quad = warp & 3;
    const int kq = e >> 2;                 // 0..3: split of the output stage's gradient components
    const int hg = kq >> 1;                // the half (and ED / FL barrier) this warp reports to
    const int cw = hg * kHalf + 64 * (kq & 1);  // first of its 64 columns
    const int row = quad * 32 + lane;
    const uint32_t t_lane = tmem + ((uint32_t)(quad * 32) << 16);
    const int n = w.n_dof;
    const uint32_t rbase = (row >> 3) * 1024 + (row & 7) * 128;
    const int r7 = row & 7;
    uint32_t* aiw_base = reinterpret_cast<uint32_t*>(gbase + kOffAiw) + e * 32;  // + slot * kEpiWarps * 32
    // per slot and tile parity (the slot's next tile is loaded while the output
    // stage of the current one is still to come): this warp's sin / cos and its
    // copy of the tile's (waypoint, first list position, length)
    float* trig_base = reinterpret_cast<float*>(gbase + kOffTrig) + e * 24;     // + (2 slot + par) * kEpiWarps * 24
    int4* tinfo_base = reinterpret_cast<int4*>(gbase + kOffTinfo) + e;           // + (2 slot + par) * kEpiWarps
    uint4* pt_base = reinterpret_cast<uint4*>(gbase + kOffPt) + row;            // + slot * kTile
    // global stash of 2 s'(z_l), layers 1..L-1 (index l - 1):
    // [slot][layer][8-column chunk][row], 16 bytes
    uint4* stash_cta = reinterpret_cast<uint4*>(w.stash) + (size_t)blockIdx.x * kSlots * (L - 1) * (kH / 8) * kTile + row;
    auto stash_at = [&](int sl, int l, int c0) -> uint4* {
      return stash_cta + ((size_t)(sl * (L - 1) + (l - 1)) * (kH / 8) + (c0 >> 3)) * kTile;
    };
    uint32_t acc_n0 = 0, acc_n1 = 0;       // ACC completions consumed per slot
    uint32_t n_out = 0;                    // output stages done (partial records)
    bool ok = true;

    // byte offset (within an A buffer) of columns c0 + 8 q .. c0 + 8 q + 7 of this row
    auto aoff = [&](int c0, int q) -> uint32_t {
      return (c0 >> 6) * (kTile * 128) + rbase + (((((c0 & 63) >> 3) + q) ^ r7) << 4);
    };
    // columns c0 .. c0 + 15 (eight FP16 / BF16 pairs) of this row
    auto store8c = [&](uint32_t abuf, int c0, const uint32_t* o) {
      if constexpr (kF8) {
        // 16 FP8 columns = one 16-byte chunk of a 128-element row
        const uint32_t off = (c0 >> 7) * (kTile * 128) + rbase + ((((c0 & 127) >> 4) ^ r7) << 4);
        ptx::st_shared_v4(abuf + off, ptx::e4m3x4(o[0], o[1]), ptx::e4m3x4(o[2], o[3]), ptx::e4m3x4(o[4], o[5]),
                          ptx::e4m3x4(o[6], o[7]));
      } else {
        ptx::st_shared_v4(abuf + aoff(c0, 0), o[0], o[1], o[2], o[3]);
        ptx::st_shared_v4(abuf + aoff(c0, 1), o[4], o[5], o[6], o[7]);
      }
    };
    // the half's epilogue is done in this warp: release the A-buffer columns it
    // wrote (and the accumulator half it read) to the even CTA's MMA issuer, one
    // arrival per warp.  Every lane's TMEM loads have completed (wait::ld) and
    // are ordered by the tcgen05 fence; its shared-memory stores are made visible
    // to the async proxy (which the tensor core reads through) before the warp
    // synchronises.
    auto arrive_lead = [&](int b) {
      ptx::tc_fence_before();
      ptx::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        if (leader) ptx::mbar_arrive(bar(base, b));
        else ptx::mbar_arrive_remote(ptx::mapa_shared(bar(base, b), 0));
      }
    };
    // tile `it` (local index) into slot it & 1: its waypoint's A_i / 2 for this
    // warp's columns and this row's point (read by its first layer), its sin /
    // cos and its list range (read by its output stage, by tile parity)
    auto load_tile = [&](int it) {
      const int sl = it & 1;
      const int tp = 2 * sl + ((it >> 1) & 1);
      const int t = 2 * (cluster + it * nclusters) + (int)rank;
      int wp = 0, start = 0, len = 0;
      if (t < ntiles) tile_lookup(w, t, wp, start, len);  // else: the odd CTA's half of the last pair tile
      if (lane == 0) tinfo_base[tp * kEpiWarps] = make_int4(wp, start, len, 0);
      float px = 0.f, py = 0.f, pz = 0.f;
      if (row < len) {
        int j;
        long long k;
        pair_at(w, wp, start + row, j, k);
        px = w.p[3 * (size_t)j];
        py = w.p[3 * (size_t)j + 1];
        pz = w.p[3 * (size_t)j + 2];
      }
      const float* Ai = w.A + (size_t)wp * kH + cw;
      uint32_t* aiw = aiw_base + sl * kEpiWarps * 32;
      float* trigw = trig_base + tp * kEpiWarps * 24;
      __syncwarp();
      // (the four warps of a row quad store the same point: each reads back its own store)
      pt_base[sl * kTile] = make_uint4(ptx::pack_f16x2(px, px), ptx::pack_f16x2(py, py), ptx::pack_f16x2(pz, pz), 0u);
      aiw[lane] = ptx::pack_f16x2(0.5f * Ai[2 * lane], 0.5f * Ai[2 * lane + 1]);
      if (lane < 2 * w.n_ang) trigw[lane] = w.trig[(size_t)wp * 2 * w.n_ang + lane];
      __syncwarp();
    };
    // h_1 = s(A_i + W_1p p) for this row and the warp's 64 columns -> the slot's
    // A buffer; 2 s'(z_1) -> the stash (the last reverse step reads it)
    auto first_layer = [&](int sl) {
      const uint32_t abuf = base + (sl ? kOffA1 : kOffA0);
      const uint32_t* aiw = aiw_base + sl * kEpiWarps * 32;
      const uint4 pt = pt_base[sl * kTile];
      uint4* st_g = fwd ? stash_cta : stash_at(sl, 1, cw);
#pragma unroll 1
      for (int cc = 0; cc < 64; cc += 16) {
        uint32_t o[8], st2[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const uint32_t u = first_layer_u2(s_w1p[(cw + cc) / 2 + i], aiw[cc / 2 + i], pt.x, pt.y, pt.z);
          if constexpr (kFmt == 0) {
            silu2_bf16(u, o[i], st2[i]);
          } else {
            uint32_t hh;
            silu2(u, hh, st2[i]);
            o[i] = to_operand<kFmt>(hh);
          }
        }
        store8c(abuf, cw + cc, o);
        if (!fwd) {
          st_g[(cc / 8) * kTile] = make_uint4(st2[0], st2[1], st2[2], st2[3]);
          st_g[(cc / 8 + 1) * kTile] = make_uint4(st2[4], st2[5], st2[6], st2[7]);
        }
      }
      arrive_lead(B_FL0 + 2 * sl + hg);
    };

    // the first tile of each slot
    for (int it = 0; it < kSlots && it < my_tiles; ++it) {
      load_tile(it);
      first_layer(it);
    }
    float fpart = 0.f;  // sum of w_o s(z_L) over this thread's 64 columns
    Schedule sc = make_sched();
    int slot, jl, s;
    while (ok && sc.next(slot, jl, s)) {
      const int it = 2 * jl + slot;
      const uint32_t abuf = base + (slot ? kOffA1 : kOffA0);
      if (s < n_steps) {
        // a reverse step starts loading the first 16 columns of its stashed factor
        // 2 s'(z_{l-1}) before it waits for the accumulator
        const int lm1 = 2 * L - 2 - s;
        const bool stashed = !fwd && s >= L - 1;
        const uint4* st_r = stashed ? stash_at(slot, lm1, cw) : stash_cta;
        uint4 dn0 = make_uint4(0u, 0u, 0u, 0u), dn1 = dn0;  // the next chunk's stash
        if (stashed) {
          dn0 = st_r[0];
          dn1 = st_r[kTile];
        }
        if (!wait_epi_warp(bar(base, B_ACC0 + slot), (slot ? acc_n1 : acc_n0) & 1u, abort_flag, tw.err)) {
          ok = false;
          break;
        }
        if (slot) ++acc_n1; else ++acc_n0;
        ptx::tc_fence_after();
        const int c0 = cw;                                         // first of this warp's 64 columns
        const uint32_t t_acc = t_lane + (uint32_t)(slot * kH) + c0;  // the slot's accumulator
        if (s < L - 2) {
          // middle forward layer l = s + 2: h_l -> A, 2 s'(z_l) -> stash
          uint4* st_g = fwd ? stash_cta : stash_at(slot, s + 2, c0);
          const float sc8 = kF8 ? tw.fp8_scale[s] : 1.f;  // FP8: the layer's weight scale
          const uint4* bh4 = reinterpret_cast<const uint4*>(s_biasH + s * (kH / 2) + (c0 >> 1));
          // 32 columns per TMEM load (one instruction, one wait), arithmetic in
          // 16-column chunks
          // both 32-column halves in one trip for BF16 operands (0.6 % faster;
          // with the first layer unrolled as well it was 0.6 % slower)
          constexpr int kMidUnroll = kFmt == 0 ? 2 : 1;
#pragma unroll kMidUnroll
          for (int cp = 0; cp < 64; cp += 32) {
            uint32_t vab[32];
            ptx::tmem_ld32(t_acc + cp, vab);
            ptx::tmem_wait_ld();
#pragma unroll
            for (int cc = cp; cc < cp + 32; cc += 16) {
              const uint32_t* v = vab + (cc - cp);
              const uint4 b0 = bh4[cc / 8], b1 = bh4[cc / 8 + 1];
              const uint32_t bh[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
              uint32_t o[8], st2[8];
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const uint32_t zp = kF8 ? ptx::pack_f16x2(sc8 * __uint_as_float(v[2 * i]), sc8 * __uint_as_float(v[2 * i + 1]))
                                        : ptx::pack_f16x2(__uint_as_float(v[2 * i]), __uint_as_float(v[2 * i + 1]));
                const uint32_t u = ptx::hfma2(zp, kHalf2, bh[i]);
                if constexpr (kFmt == 0) {
                  silu2_bf16(u, o[i], st2[i]);
                } else {
                  uint32_t hh;
                  silu2(u, hh, st2[i]);
                  o[i] = to_operand<kFmt>(hh);
                }
              }
              store8c(abuf, c0 + cc, o);
              if (!fwd) {
                st_g[(cc / 8) * kTile] = make_uint4(st2[0], st2[1], st2[2], st2[3]);
                st_g[(cc / 8 + 1) * kTile] = make_uint4(st2[4], st2[5], st2[6], st2[7]);
              }
            }
          }
        } else if (s == L - 2) {
          // last forward layer: f partial (FP32 sum), g_L = w_o s'(z_L) -> A
          fpart = 0.f;
          const float sc8 = kF8 ? tw.fp8_scale[L - 2] : 1.f;
          const uint4* bh4 = reinterpret_cast<const uint4*>(s_biasH + (L - 2) * (kH / 2) + (c0 >> 1));
          // two chunks per trip for BF16 operands (0.4 % faster; FP16 0.6 % slower)
          constexpr int kLastUnroll = kFmt == 0 ? 2 : 1;
#pragma unroll kLastUnroll
          for (int cc = 0; cc < 64; cc += 16) {
            uint32_t v[16];
            ptx::tmem_ld16(t_acc + cc, v);
            const uint4 b0 = bh4[cc / 8], b1 = bh4[cc / 8 + 1];
            const uint32_t bh[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
            const uint4* wh4 = reinterpret_cast<const uint4*>(s_woh + (c0 + cc) / 2);
            const uint4 w0 = wh4[0], w1 = wh4[1];
            const uint32_t wh[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
            ptx::tmem_wait_ld();
            uint32_t o[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const uint32_t zp = kF8 ? ptx::pack_f16x2(sc8 * __uint_as_float(v[2 * i]), sc8 * __uint_as_float(v[2 * i + 1]))
                                      : ptx::pack_f16x2(__uint_as_float(v[2 * i]), __uint_as_float(v[2 * i + 1]));
              const uint32_t u = ptx::hfma2(zp, kHalf2, bh[i]);
              const float2 wo = *reinterpret_cast<const float2*>(s_wo + c0 + cc + 2 * i);
              if constexpr (kFmt == 0) {
                // s(z) = u (1 + t) exactly in FP32 for f; g_L = (w_o / 2) 2 s'(z)
                // exactly in FP32, rounded once to BF16
                const uint32_t t = ptx::htanh2(u);
                const uint32_t tp1 = ptx::hadd2(kOne2, t);
                float h0, h1, g0, g1;
                ptx::f16x2_products(u, tp1, h0, h1);
                fpart = fmaf(wo.x, h0, fmaf(wo.y, h1, fpart));
                ptx::f16x2_products(wh[i], ptx::hfma2(tp1, ptx::hfnms2(u, t), tp1), g0, g1);
                o[i] = ptx::pack_bf16x2(g0, g1);
              } else {
                uint32_t hh, s2;
                silu2(u, hh, s2);
                fpart = fmaf(wo.x, ptx::f16lo(hh), fmaf(wo.y, ptx::f16hi(hh), fpart));
                o[i] = to_operand<kFmt>(ptx::hmul2(wh[i], s2));
              }
            }
            if (!fwd) store8c(abuf, c0 + cc, o);
          }
          s_f[((2 * slot + (jl & 1)) * 4 + kq) * kTile + row] = fpart;
          ptx::mbar_arrive(bar(base, B_FD0 + slot));
        } else {
          // reverse step: g_{l-1} = acc * 2 s'(z_{l-1}), acc = (W_l^T / 2) g_l
          // FP8: acc = (64 / s_rev) (W^T / 2) g, so acc * s_rev is the next
          // operand already carrying its x64
          const float sc8 = kF8 ? tw.fp8_scale[L - 1 + (2 * L - 3 - s)] : 1.f;
#pragma unroll
          for (int cc = 0; cc < 64; cc += 16) {
            uint32_t v[16], d2[8];
            ptx::tmem_ld16(t_acc + cc, v);
            d2[0] = dn0.x; d2[1] = dn0.y; d2[2] = dn0.z; d2[3] = dn0.w;
            d2[4] = dn1.x; d2[5] = dn1.y; d2[6] = dn1.z; d2[7] = dn1.w;
            if (cc + 16 < 64) {
              dn0 = st_r[((cc + 16) / 8) * kTile];
              dn1 = st_r[((cc + 16) / 8 + 1) * kTile];
            }
            ptx::tmem_wait_ld();
            uint32_t o[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              if constexpr (kFmt == 0) {
                // BF16: the product in FP32, one rounding to BF16 (one pack instead of two)
                o[i] = ptx::pack_bf16x2(__uint_as_float(v[2 * i]) * ptx::f16lo(d2[i]),
                                        __uint_as_float(v[2 * i + 1]) * ptx::f16hi(d2[i]));
              } else {
                const uint32_t ap = kF8 ? ptx::pack_f16x2(sc8 * __uint_as_float(v[2 * i]), sc8 * __uint_as_float(v[2 * i + 1]))
                                        : ptx::pack_f16x2(__uint_as_float(v[2 * i]), __uint_as_float(v[2 * i + 1]));
                o[i] = to_operand<kFmt>(ptx::hmul2(ap, d2[i]));
              }
            }
            store8c(abuf, c0 + cc, o);
          }
        }
        // (forward-only: the last step produces no operand, so no MMA waits for it)
        if (!(fwd && s == n_steps - 1)) arrive_lead(B_ED0 + 2 * slot + hg);
        // after the tile's last reverse step: fetch the slot's next tile, whose
        // first layer the tail writes as soon as the Jacobian chain has read the
        // A buffer (this step has slack; the tail does not)
        if (!fwd && s == n_steps - 1 && it + kSlots < my_tiles) load_tile(it + kSlots);
        continue;
      }

      // ---- tail item of the slot's tile -------------------------------------------
      const int4 ti = tinfo_base[(2 * slot + (jl & 1)) * kEpiWarps];
      const int cur_wp = ti.x, cur_start = ti.y, cur_len = ti.z;
      const bool more = it + kSlots < my_tiles;
      if (fwd) {
        // the next tile of the slot can start at once: the last step's MMAs have
        // completed (its accumulator was read) and no MMA reads the A buffer
        if (more) {
          load_tile(it + kSlots);
          first_layer(slot);
        }
        if (!wait_epi_warp(bar(base, B_FD0 + slot), (uint32_t)jl & 1u, abort_flag, tw.err)) { ok = false; break; }
        if (kq == 0 && row < cur_len) {
          int j;
          long long k;
          pair_at(w, cur_wp, cur_start + row, j, k);
          const float* sf = s_f + (2 * slot + (jl & 1)) * 4 * kTile;
          w.f_out[k] = sf[row] + sf[kTile + row] + sf[2 * kTile + row] + sf[3 * kTile + row] + tw.bout;
        }
        continue;
      }
      // the input-Jacobian chain of this tile (it has read the A buffer)
      if (!wait_epi_warp(bar(base, B_ACCJ0 + slot), (uint32_t)jl & 1u, abort_flag, tw.err)) { ok = false; break; }
      ptx::tc_fence_after();
      // the 4 warps of a row quad split the gradient components (d = kq, kq + 4,
      // kq + 8) and each reads only the Jacobian columns they need (warp-uniform
      // columns, no indexed registers), and the sin / cos they need, before the
      // next tile replaces them
      uint32_t jv[3][2];
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const int d = kq + 4 * m;
        ptx::tmem_ld2(t_lane + (uint32_t)(slot * kH + kHalf) + (d < 2 ? 0 : 2 * d - 2), jv[m]);
      }
      float trs[3], trc[3];
      {
        const float* tr = trig_base + (2 * slot + (jl & 1)) * kEpiWarps * 24;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          const int a = kq + 4 * m - 2;
          trs[m] = (a >= 0 && a < w.n_ang) ? tr[2 * a] : 0.f;
          trc[m] = (a >= 0 && a < w.n_ang) ? tr[2 * a + 1] : 0.f;
        }
      }
      ptx::tmem_wait_ld();
      // the slot's next tile: its first layer goes into the A buffer (free: the
      // Jacobian chain has completed) and its first MMAs into the accumulator
      // (free: the Jacobian columns were just read, ordered by the arrival)
      if (more) first_layer(slot);  // its inputs were loaded after the last reverse step
      // output stage, shared by all 16 warps
      if (!wait_epi_warp(bar(base, B_FD0 + slot), (uint32_t)jl & 1u, abort_flag, tw.err)) { ok = false; break; }
      const float* sf = s_f + (2 * slot + (jl & 1)) * 4 * kTile;
      const float fval = sf[row] + sf[kTile + row] + sf[2 * kTile + row] + sf[3 * kTile + row] + tw.bout;
      if (kF8) {  // J = (s_J / 64) x the accumulator of FP8 W_1q^T and the x64 operand
        const float js = tw.fp8_scale[2 * L - 2] * (1.f / kGradScale8);
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          jv[m][0] = __float_as_uint(js * __uint_as_float(jv[m][0]));
          jv[m][1] = __float_as_uint(js * __uint_as_float(jv[m][1]));
        }
      }
      float dqm[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const int d = kq + 4 * m;
        if (d < 2) {
          dqm[m] = __uint_as_float(d == 0 ? jv[m][0] : jv[m][1]);
        } else if (d < n) {  // angle a = d - 2: (sin, cos) chain rule of Eq. (10)
          dqm[m] = trc[m] * __uint_as_float(jv[m][0]) - trs[m] * __uint_as_float(jv[m][1]);
        } else {
          dqm[m] = 0.f;
        }
      }
      const bool valid = row < cur_len;
      int j = -1;
      long long k = 0;
      if (valid) pair_at(w, cur_wp, cur_start + row, j, k);
      if (w.mode == kQuery) {
        if (valid) {
          if (kq == 0) w.f_out[k] = fval;
          if (w.g_out) {
            float* go = w.g_out + (size_t)k * n;
#pragma unroll
            for (int m = 0; m < 3; ++m)
              if (kq + 4 * m < n) go[kq + 4 * m] = dqm[m];
          }
        }
      } else {
        // the merge warp has read the previous tile's records
        if (n_out > 0 && !wait_epi_warp(bar(base, B_MD), (n_out - 1u) & 1u, abort_flag, tw.err)) {
          ok = false;
          break;
        }
        warp_partial_part(w.mode, w.param, valid, fval, dqm, kq, n, j, cur_start + row, &s_part[quad]);
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(bar(base, B_PD));
        ++n_out;
      }
    }
  }

  // ---- teardown ---------------------------------------------------------------
  // every thread of both CTAs gets here (all waits are bounded): no CTA leaves
  // while its peer may still signal its barriers or read its operands
  ptx::tc_fence_before();
  ptx::cluster_sync();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc_pair(tmem, kTmemCols);
  }
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// Row-major operand image, 128-byte swizzled boxes of one 128-byte row width
// (64 16-bit or 128 FP8 elements) by box_rows rows.
int encode_2d(CUtensorMap* m, const void* ptr, int rows, int cols, int box_rows, int fmt) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return 1;
  const int eb = fmt == 2 ? 1 : 2;
  cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)cols * eb};
  cuuint32_t box[2] = {(cuuint32_t)(128 / eb), (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  const CUtensorMapDataType dt = fmt == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                 : (fmt == 1 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
  CUresult r = enc(m, dt, 2,
                   const_cast<void*>(ptr), gdim, gstride, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : 2;
}

uint16_t to_bits(float x, bool f16) {
  if (f16) {
    const __half h = __float2half_rn(x);
    return *reinterpret_cast<const uint16_t*>(&h);
  }
  const __nv_bfloat16 b = __float2bfloat16_rn(x);
  return *reinterpret_cast<const uint16_t*>(&b);
}

}  // namespace

int tc_tile_pairs() { return kTile; }

// [slot][layer 1..L-1][8-column chunk][row] of 16 bytes per CTA
static size_t stash_bytes_per_cta(int L) { return L >= 2 ? (size_t)kSlots * (L - 1) * (kH / 8) * kTile * 16 : 0; }

size_t tc_stash_bytes(int L, int num_sms) { return stash_bytes_per_cta(L) * (size_t)(num_sms > 1 ? num_sms : 2); }

bool tc_supported(int H, int L, int n_dof) { return H == kH && L >= 2 && L <= 4 && n_dof >= 3 && n_dof <= kMaxDof; }

// the input-Jacobian chain is one MMA of N = 32 (16 rows per CTA of the pair):
// d_q = 2 n_dof - 2 <= 22 for every supported n_dof, zero rows pad
int tc_nj(int) { return 32; }

// Image layout (16-bit, row-major, 256 columns): rows [256 m, 256 m + 256) hold
// W_{m+2} for m = 0..L-2 (forward operands, row = output feature), then rows
// [256 (L-1+m), ...) hold W_{m+2}^T / 2 (reverse operands, row = input
// feature; the factor 1/2 is exact), then nj rows of W_1q^T (row d = input
// column 3 + d of layer 1; zero rows pad).
size_t tc_image_elems(int H, int L, int d_q) {
  return (size_t)2 * (L - 1) * H * H + (size_t)tc_nj(d_q) * H;
}

uint8_t to_e4m3(float x) { return (uint8_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3); }

float max_abs(const float* x, size_t n, size_t stride) {
  float m = 0.f;
  for (size_t i = 0; i < n; ++i) m = fmaxf(m, fabsf(x[i * stride]));
  return m;
}

void tc_build_image(const float* W, int H, int L, int d_q, int d_in, int fmt, void* out_v, float* scales) {
  const bool f8 = fmt == 2;
  uint16_t* out = static_cast<uint16_t*>(out_v);
  uint8_t* out8 = static_cast<uint8_t*>(out_v);
  size_t off = (size_t)H * d_in + H;
  for (int m = 0; m < L - 1; ++m) {
    const float* Wl = W + off;
    const size_t f0 = (size_t)m * H * H, r0 = (size_t)(L - 1 + m) * H * H;
    // FP8: W_l = s W8 with s = max |W_l| / 448; the reverse operand W_l^T / 2
    // uses the same bytes transposed with scale s / 2
    float sc = 1.f;
    if (f8) {
      const float mx = max_abs(Wl, (size_t)H * H, 1);
      sc = mx > 0.f ? mx / 448.f : 1.f;
      scales[m] = sc;
      scales[L - 1 + m] = 0.5f * sc;
    }
    for (int o = 0; o < H; ++o)
      for (int i = 0; i < H; ++i) {
        const float v = Wl[(size_t)o * H + i];
        if (f8) {
          const uint8_t b = to_e4m3(v / sc);
          out8[f0 + (size_t)o * H + i] = b;
          out8[r0 + (size_t)i * H + o] = b;
        } else {
          out[f0 + (size_t)o * H + i] = to_bits(v, fmt == 1);
          out[r0 + (size_t)i * H + o] = to_bits(0.5f * v, fmt == 1);
        }
      }
    off += (size_t)H * H + H;
  }
  const size_t j0 = (size_t)2 * (L - 1) * H * H;
  const int nj = tc_nj(d_q);
  float js = 1.f;
  if (f8) {
    float mx = 0.f;
    for (int d = 0; d < d_q; ++d) mx = fmaxf(mx, max_abs(W + 3 + d, (size_t)H, (size_t)d_in));
    js = mx > 0.f ? mx / 448.f : 1.f;
    scales[2 * (L - 1)] = js;
  }
  for (int d = 0; d < nj; ++d)
    for (int c = 0; c < H; ++c) {
      const float v = d < d_q ? W[(size_t)c * d_in + 3 + d] : 0.f;
      if (f8) out8[j0 + (size_t)d * H + c] = to_e4m3(v / js);
      else out[j0 + (size_t)d * H + c] = to_bits(v, fmt == 1);
    }
}

int tc_encode_maps(const void* image, int H, int L, int d_q, int fmt, TcWeights& tw) {
  // boxes: one CTA's share of a chain (kRowsCta weight rows, nj / 2 Jacobian rows) x 128 bytes
  int rc = encode_2d(&tw.map_w, image, 2 * (L - 1) * H, H, kRowsCta, fmt);
  if (rc) return rc;
  const size_t eb = fmt == 2 ? 1 : 2;
  return encode_2d(&tw.map_j, static_cast<const uint8_t*>(image) + (size_t)2 * (L - 1) * H * H * eb, tc_nj(d_q), H,
                   tc_nj(d_q) / 2, fmt);
}

template <int kFmt, bool kFwd>
cudaError_t launch_tc_t(const WorkDesc& w, const TcWeights& tw, int num_sms, cudaStream_t s) {
  // clusters of 2 CTAs (one per SM); as many as can be resident at once, each
  // looping over pair tiles
  static int max_clusters[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  const bool cached = dev >= 0 && dev < 64;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = kSmemBytes;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int mc = cached ? max_clusters[dev] : 0;
  if (mc <= 0) {
    cudaError_t e = cudaFuncSetAttribute(tc_fused_kernel<kFmt, kFwd>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSmemBytes);
    if (e != cudaSuccess) return e;
    cfg.gridDim = dim3(2);
    e = cudaOccupancyMaxActiveClusters(&mc, (void*)tc_fused_kernel<kFmt, kFwd>, &cfg);
    if (e != cudaSuccess) return e;
    if (mc <= 0) return cudaErrorLaunchOutOfResources;
    if (cached) max_clusters[dev] = mc;
  }
  if (num_sms > 0 && 2 * mc > num_sms) mc = num_sms / 2 > 0 ? num_sms / 2 : 1;
  const int npt = (w.n_tiles + 1) / 2;
  if (npt <= 0) return cudaSuccess;
  const int grid = 2 * (npt < mc ? npt : mc);
  cfg.gridDim = dim3(grid);
  const size_t stash_bytes = kFwd ? 0 : stash_bytes_per_cta(tw.L) * (size_t)grid;
  if (stash_bytes == 0 || w.stash != nullptr)
    return cudaLaunchKernelEx(&cfg, tc_fused_kernel<kFmt, kFwd>, w, tw.map_w, tw.map_j, tw);
  // the stash from the library's pool, stream-ordered around the launch
  WorkDesc ws = w;
  cudaError_t e = lib_malloc_async(&ws.stash, stash_bytes, s);
  if (e != cudaSuccess) return e;
  e = cudaLaunchKernelEx(&cfg, tc_fused_kernel<kFmt, kFwd>, ws, tw.map_w, tw.map_j, tw);
  const cudaError_t ef = cudaFreeAsync(ws.stash, s);
  return e != cudaSuccess ? e : ef;
}

cudaError_t launch_wait_expiry_probe(int* err, long long limit_cycles, int* seen, cudaStream_t s) {
  wait_expiry_probe_kernel<<<1, 64, 0, s>>>(err, limit_cycles, seen);
  return cudaGetLastError();
}

cudaError_t launch_tc(const WorkDesc& w, const TcWeights& tw, int num_sms, cudaStream_t s) {
  if (w.mode == kQuery && w.g_out == nullptr) {
    if (tw.fmt == 2) return launch_tc_t<2, true>(w, tw, num_sms, s);
    return tw.fmt == 1 ? launch_tc_t<1, true>(w, tw, num_sms, s) : launch_tc_t<0, true>(w, tw, num_sms, s);
  }
  if (tw.fmt == 2) return launch_tc_t<2, false>(w, tw, num_sms, s);
  return tw.fmt == 1 ? launch_tc_t<1, false>(w, tw, num_sms, s) : launch_tc_t<0, false>(w, tw, num_sms, s);
}

}  // namespace gcdf
