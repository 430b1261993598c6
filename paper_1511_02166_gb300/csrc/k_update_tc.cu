// k_update_tc.cu -- the trailing update A22 -= L21 U12 of the step-synchronous
// blocked LU of large airfoils (k_lu_large.cu) on the 5th-generation tensor
// cores: tcgen05.mma (kind::tf32) with the accumulator in tensor memory, the
// operands loaded by the tensor memory access (TMA) unit and the result added
// into A22 by TMA reduce-add.
//
// The factor is in the tiled layout of tl_layout.cuh: every 128 x 32 chunk of
// a full tile is 128 rows of 128 bytes on a 128-byte boundary of the factor
// buffer, so one two-dimensional tensor map (the whole buffer as rows of 32
// floats, 128-byte swizzle) describes every operand chunk of every airfoil.
// At step K >= 1 the output tile (I, J) (I, J > K) takes A = L21 tile (I, K)
// (rows x k: K-major) and B = U12 tile (K, J), which k_large_trsm stored
// transposed (columns x k: K-major as well), four chunks of K = 32 each.  At
// step 0 the inner dimension is the ragged first block (e <= 128 columns of
// L, e rows of U, neither on a 16-byte grid): the converter warps load those
// operands themselves, zero-padded to whole chunks.
//
// One block takes 128 x 128 output tiles of one airfoil (block y of gridDim.y
// strides over the airfoil's tiles).  Warp-specialised, 320 threads:
//   warp 8     one lane issues the TMA loads of a chunk of A and of B into a
//              shared-memory stage (three stages, 64 KB each);
//   warps 4-7  converters: split each operand value x = x_hi + x_lo, x_hi = x
//              rounded to TF32 (in place), x_lo = x - x_hi (exact in FP32,
//              into the stage's second half); at step 0 they first load it;
//   warp 9     one lane issues the MMAs: A_hi B_hi + A_hi B_lo + A_lo B_hi
//              ("3xTF32", the dropped A_lo B_lo is ~2^-22 relative; TF32 alone
//              would make the factor far less accurate than FP32 and the
//              refinement would stall on these ill-conditioned systems),
//              M = N = 128, K = 8 per instruction, into one of two FP32
//              accumulators in tensor memory (2 x 128 columns);
//   warps 0-3  epilogue: read a finished accumulator (warp w owns TMEM lanes
//              = tile rows 32w..32w+31), write -D in 128 x 32 chunks into a
//              swizzled staging buffer, and let the TMA add it to A22
//              (cp.reduce.async.bulk.tensor .add: the read-modify-write of
//              A22 happens in L2, not in the block).
// Full (TMA bytes) / converted / empty (MMA commit) mbarriers connect the
// stages, full / empty mbarriers the accumulators; the epilogue of one tile
// overlaps the MMAs of the next.
//
// Every pipeline wait is bounded (`spin` polls, a kernel argument) and polls a
// shared failure flag: a block that gives up stops issuing work, and every
// role leaves its loop.  Before the block ends, the TMA lane waits for the
// loads it has issued, the epilogue for its reduce-adds, and the block for a
// final arrival that the MMA lane commits on every path after the last MMA it
// issued; these waits have their own bound (kDoneLimit) and ignore the flag,
// so that nothing still writes shared or tensor memory when the block sets
// info[b] = PANEL_INFO_DEVICE_TIMEOUT, frees its tensor memory and returns.
#include <cudaTypedefs.h>

#include <mutex>

#include "tl_layout.cuh"

namespace panel {

namespace {

constexpr int kTM = 128;                                // tile rows (MMA M)
constexpr int kTN = 128;                                // tile columns (MMA N)
constexpr int kKC = kTlC;                               // K per chunk (32)
constexpr int kStages = 3;
constexpr uint32_t kOpBytes = kTM * kKC * 4;            // one operand chunk: 16 KB
constexpr uint32_t kStageBytes = 4 * kOpBytes;          // A (-> A_hi), A_lo, B (-> B_hi), B_lo
constexpr uint32_t kEpiBytes = kOpBytes;                // a 128 x 32 chunk of -D
constexpr int kEpiBufs = 2;
constexpr uint32_t kBarOff = kStages * kStageBytes + kEpiBufs * kEpiBytes;
constexpr uint32_t kSmemBytes = kBarOff + 256 + 1024;   // barriers, then 1 KB alignment slack
constexpr uint32_t kTmemCols = 2 * kTN;                 // two FP32 accumulators, 128 x 128 each
constexpr int kThreadsTc = 320;
constexpr int kWarpTma = 8, kWarpMma = 9;
// bound of the final waits for the block's own asynchronous operations (they
// finish in microseconds; the bound only keeps the wait finite)
constexpr long long kDoneLimit = 1ll << 24;

// Instruction descriptor, kind::tf32: D = F32 (bits 4-5 = 1), A = B = TF32
// (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22,
// M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);

// Shared-memory matrix descriptor of a K-major operand with the 128-byte
// swizzle (the layout the TMA writes with CU_TENSOR_MAP_SWIZZLE_128B): rows of
// 128 bytes, 8-row atoms of 1 KB (stride byte offset 1024), leading byte
// offset unused (1); start address >> 4 in bits 0-13, descriptor version 1
// (bit 46), layout type 2 = 128-byte swizzle (bits 61-63).  Stepping K by 8
// TF32 values inside the atom adds 32 bytes to the start address.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) |
         (1ull << 46) | (2ull << 61);
}

// Byte offset of element (row, k) of a 128 x 32 operand chunk in the 128-byte
// swizzled layout: 16-byte units of a row XOR the row's position in its atom.
__device__ __forceinline__ uint32_t sw_off(int row, int k) {
  return (uint32_t)(row * 128 + ((((k >> 2) ^ (row & 7)) & 7) << 4) + ((k & 3) << 2));
}

__device__ __forceinline__ float tf32_hi(float x) {
  // round to the nearest TF32 value (ties away), low 13 mantissa bits cleared
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// Waits for the phase with the given parity; false if `spin` polls ran out
// (then sets *fail) or another thread of the block has already given up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* fail,
                                          long long spin) {
  for (long long it = 0; it < spin; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255) == 255 && *fail) return false;
  }
  *fail = 1;
  return false;
}

// A final wait for the block's own asynchronous operations: bounded, but it
// does not give up when *fail is set (what was issued before is still running).
__device__ __forceinline__ bool mbar_wait_done(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < kDoneLimit; ++it)
    if (mbar_try(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap* map, int y,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_reduce_add(const CUtensorMap* map, int y, uint32_t src) {
  asm volatile(
      "cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group "
      "[%0, {%1, %2}], [%3];" ::"l"(reinterpret_cast<uint64_t>(map)),
      "r"(0), "r"(y), "r"(src)
      : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

__device__ __forceinline__ void bulk_wait_read_1() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}

__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// True on every epilogue thread iff `ok` holds on all 128 of them (named
// barrier 1 with an AND reduction): the epilogue leaves its loop together.
__device__ __forceinline__ bool epi_all(bool ok) {
  uint32_t all;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.and.pred p, 1, 128, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(all)
      : "r"((uint32_t)ok)
      : "memory");
  return all != 0;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace

__global__ void __launch_bounds__(kThreadsTc, 1)
    k_update_tc(SolveArgs a, const __grid_constant__ CUtensorMap tmap, int K, long long spin) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  const Batch& bt = a.bt;
  const int b = bt.order[blockIdx.x];
  const int n = airfoil_n(bt, b), m = n + 1;
  if (!(m > kLargeM && n <= bt.n_max && a.info[b] == 0)) return;
  TlGeom g;
  g.init(m, bt.mat_off[b]);
  if (K >= g.T - 1) return;
  const int nt = g.T - 1 - K, tiles = nt * nt;
  if ((int)blockIdx.y >= tiles) return;
  const int nkc = (K == 0) ? (g.e + kKC - 1) / kKC : kTlB / kKC;
  const int my_tiles = (tiles - (int)blockIdx.y + (int)gridDim.y - 1) / (int)gridDim.y;
  const int nq = my_tiles * nkc;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sraw = smem_u32(smraw);
  const uint32_t sbase = (sraw + 1023u) & ~1023u;
  unsigned char* gbase = smraw + (sbase - sraw);
  const uint32_t ebase = sbase + kStages * kStageBytes;
  const uint32_t bar_base = sbase + kBarOff;
  // full[3] conv[3] empty[3] tfull[2] tempty[2] done
  auto full_bar = [&](int st) { return bar_base + 8u * st; };
  auto conv_bar = [&](int st) { return bar_base + 8u * (kStages + st); };
  auto empty_bar = [&](int st) { return bar_base + 8u * (2 * kStages + st); };
  auto tfull_bar = [&](int ac) { return bar_base + 8u * (3 * kStages + ac); };
  auto tempty_bar = [&](int ac) { return bar_base + 8u * (3 * kStages + 2 + ac); };
  const uint32_t done_bar = bar_base + 8u * (3 * kStages + 4);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(gbase + kBarOff + 128);
  volatile int* fail = reinterpret_cast<volatile int*>(gbase + kBarOff + 132);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int st = 0; st < kStages; ++st) {
      mbar_init(full_bar(st), 1);   // the TMA lane's arrival (+ the bytes of two chunks)
      mbar_init(conv_bar(st), 4);   // one arrival per converter warp
      mbar_init(empty_bar(st), 1);  // tcgen05.commit
    }
    for (int ac = 0; ac < 2; ++ac) {
      mbar_init(tfull_bar(ac), 1);   // tcgen05.commit
      mbar_init(tempty_bar(ac), 4);  // one arrival per epilogue warp
    }
    mbar_init(done_bar, 1);
    *fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const float* F = a.LU + bt.mat_off[b];

  auto tile_ij = [&](int tau, int& I, int& J) {
    const int t = (int)blockIdx.y + tau * (int)gridDim.y;
    I = K + 1 + t / nt;
    J = K + 1 + t % nt;
  };
  // row of the tensor map (rows of 32 floats) where chunk kc of tile (I, J) starts
  auto map_row = [&](int I, int J, int kc) {
    return (int)((g.base + g.tile(I, J) + (int64_t)kc * kTlChunk) >> 5);
  };

  if (warp == kWarpTma) {
    // ---------------- TMA loads (one lane) ----------------
    if (lane == 0) {
      int issued = 0;
      for (int q = 0; q < nq; ++q) {
        const int st = q % kStages, u = q / kStages;
        if (u >= 1 && !mbar_wait(empty_bar(st), (u - 1) & 1, fail, spin)) break;
        if (K == 0) {  // the converters load the ragged operands themselves
          mbar_arrive(full_bar(st));
          continue;
        }
        int I, J;
        tile_ij(q / nkc, I, J);
        const int kc = q % nkc;
        const uint32_t sA = sbase + st * kStageBytes;
        mbar_arrive_tx(full_bar(st), 2 * kOpBytes);
        tma_load(sA, &tmap, map_row(I, K, kc), full_bar(st));
        tma_load(sA + 2 * kOpBytes, &tmap, map_row(K, J, kc), full_bar(st));
        issued = q + 1;
      }
      // the loads still in flight land before the block may end
      for (int q = max(0, issued - kStages); q < issued; ++q)
        mbar_wait_done(full_bar(q % kStages), (q / kStages) & 1);
    }
    __syncwarp();
  } else if (warp >= 4 && warp < 8) {
    // ---------------- converters: x -> (x_hi in place, x_lo) ----------------
    const int ct = tid - 128;
    constexpr int kPer = kTM * kKC / 128;  // operand values of a chunk per converter thread
    for (int q = 0; q < nq; ++q) {
      const int st = q % kStages, u = q / kStages;
      // step 0: this thread's values of the chunk, all loads in flight before
      // the stage is waited for.  A: rows ct / 32 + 4 j of the ragged tile
      // (I, 0), column k0 + ct % 32; B: row k0 + j of block row 0 (row-major),
      // column c0 + ct.  A warp reads 128 contiguous bytes per load.
      float va[kPer], vb[kPer];
      if (K == 0) {
        int I, J;
        tile_ij(q / nkc, I, J);
        const int k0 = (q % nkc) * kKC, c0 = g.start(J);
        const int ak = ct & 31, ar0 = ct >> 5;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
          va[j] = (k0 + ak < g.e) ? F[g.rag(I, ar0 + 4 * j, k0 + ak)] : 0.0f;
          vb[j] = (k0 + j < g.e) ? F[(int64_t)(k0 + j) * m + c0 + ct] : 0.0f;
        }
      }
      // every lane waits (acquiring the TMA's bytes), and the warp leaves together
      const bool ok = mbar_wait(full_bar(st), u & 1, fail, spin);
      if (!__all_sync(0xffffffffu, ok)) break;
      unsigned char* S = gbase + st * kStageBytes;
      if (K == 0) {
        const int ak = ct & 31, ar0 = ct >> 5;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
          const uint32_t oa = sw_off(ar0 + 4 * j, ak);
          const float ha = tf32_hi(va[j]);
          *reinterpret_cast<float*>(S + oa) = ha;
          *reinterpret_cast<float*>(S + kOpBytes + oa) = va[j] - ha;
          const uint32_t ob = sw_off(ct, j);
          const float hb = tf32_hi(vb[j]);
          *reinterpret_cast<float*>(S + 2 * kOpBytes + ob) = hb;
          *reinterpret_cast<float*>(S + 3 * kOpBytes + ob) = vb[j] - hb;
        }
      } else {
        float4* A4 = reinterpret_cast<float4*>(S);
        float4* B4 = reinterpret_cast<float4*>(S + 2 * kOpBytes);
        constexpr int kVec = kOpBytes / 16;  // float4 per chunk
#pragma unroll 4
        for (int j = 0; j < kVec / 128; ++j) {
          const int i = ct + 128 * j;
          const float4 va = A4[i], vb = B4[i];
          const float4 ha = make_float4(tf32_hi(va.x), tf32_hi(va.y), tf32_hi(va.z),
                                        tf32_hi(va.w));
          const float4 hb = make_float4(tf32_hi(vb.x), tf32_hi(vb.y), tf32_hi(vb.z),
                                        tf32_hi(vb.w));
          A4[i] = ha;
          A4[kVec + i] = make_float4(va.x - ha.x, va.y - ha.y, va.z - ha.z, va.w - ha.w);
          B4[i] = hb;
          B4[kVec + i] = make_float4(vb.x - hb.x, vb.y - hb.y, vb.z - hb.z, vb.w - hb.w);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(conv_bar(st));
    }
  } else if (warp == kWarpMma) {
    // ---------------- MMA issue (one lane) ----------------
    if (lane == 0) {
      for (int q = 0; q < nq; ++q) {
        const int st = q % kStages, u = q / kStages;
        const int kc = q % nkc, tau = q / nkc, ac = tau & 1, v = tau >> 1;
        if (kc == 0 && v >= 1 && !mbar_wait(tempty_bar(ac), (v - 1) & 1, fail, spin)) break;
        if (!mbar_wait(conv_bar(st), u & 1, fail, spin)) break;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(ac * kTN);
        const uint32_t ah = sbase + st * kStageBytes, al = ah + kOpBytes;
        const uint32_t bh = ah + 2 * kOpBytes, bl = ah + 3 * kOpBytes;
#pragma unroll
        for (int s = 0; s < kKC / 8; ++s) {  // K = 8 per MMA: 32 bytes of each row
          const uint32_t ko = 32u * s;
          const uint32_t acc0 = (kc > 0 || s > 0) ? 1u : 0u;
          tc_mma(d, desc_sw128(ah + ko), desc_sw128(bh + ko), acc0);
          tc_mma(d, desc_sw128(ah + ko), desc_sw128(bl + ko), 1u);
          tc_mma(d, desc_sw128(al + ko), desc_sw128(bh + ko), 1u);
        }
        tc_commit(empty_bar(st));
        if (kc == nkc - 1) tc_commit(tfull_bar(ac));
      }
      tc_commit(done_bar);  // arrives once every MMA issued above has completed
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: A22 += -D by TMA reduce-add ----------------
    const int r = 32 * warp + lane;  // tile row = TMEM lane
    int cnt = 0;
    for (int tau = 0; tau < my_tiles; ++tau) {
      const int ac = tau & 1, v = tau >> 1;
      if (!epi_all(mbar_wait(tfull_bar(ac), v & 1, fail, spin))) break;
      tc_fence_after();
      int I, J;
      tile_ij(tau, I, J);
#pragma unroll 1
      for (int s = 0; s < kTN / kKC; ++s) {
        float v32[32];
        tc_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(ac * kTN + kKC * s), v32);
        if (s == kTN / kKC - 1) {  // the accumulator is free once its last columns are read
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(tempty_bar(ac));
        }
        const uint32_t buf = (uint32_t)(cnt & 1) * kEpiBytes;
        if (tid == 0 && cnt >= 2) bulk_wait_read_1();  // this buffer's previous reduce has read it
        epi_bar();
        unsigned char* E = gbase + kStages * kStageBytes + buf;
#pragma unroll
        for (int j = 0; j < 8; ++j)
          *reinterpret_cast<float4*>(E + r * 128 + (((j ^ (r & 7)) & 7) << 4)) =
              make_float4(-v32[4 * j], -v32[4 * j + 1], -v32[4 * j + 2], -v32[4 * j + 3]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        epi_bar();
        if (tid == 0) tma_reduce_add(&tmap, map_row(I, J, s), ebase + buf);
        ++cnt;
      }
    }
    if (tid == 0) bulk_wait_all();  // every reduce-add has completed
  }

  // every MMA this block issued has completed once done_bar has flipped (the
  // MMA lane commits it on every path, also after giving up)
  __syncthreads();
  const bool drained = mbar_wait_done(done_bar, 0);
  if (!drained || *fail) {
    if (tid == 0) a.info[b] = PANEL_INFO_DEVICE_TIMEOUT;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// k_trsm_tc -- the triangular solves of step K >= 1 on the tensor cores:
//   L21 = A21 U11^{-1}  for the tiles (I, K), I > K   (blocks with y odd);
//   U12 = L11^{-1} A12  for the tiles (K, J), J > K   (blocks with y even),
// written back in place, U12 transposed (the update's K-major B operand).
// In MMA terms D[M][N] = sum_k A[M][k] B[N][k] with M = 128 rows of the tile
// (r of A21, or c of A12^T), N = t, B[t][k] = X[k][t] for X = U11^{-1} (L21)
// or B[t][k] = L11^{-1}[t][k] (U12^T).  Per block:
//   1. the diagonal tile (K, K) is staged and the one triangular inverse this
//      block needs is formed by 32 x 32 blocks (the diagonal blocks by
//      substitution in registers, then the blocks below them as small products,
//      operands read as broadcast vector loads); it is split into TF32 hi / lo
//      and kept in shared memory as the B operand of all the block's tiles
//      (128 KB);
//   2. the tiles stream through three stages of 32 KB: warp 8 loads a K-chunk
//      by TMA (a 128 x 32 chunk of A21, or four 32 x 32 boxes of A12, each of
//      which a converter warp transposes to rows of A12^T in place: a box and
//      its swizzled image are the same 4 KB), warps 4-7 split it into hi (in
//      place) and lo, warp 9 issues the 3xTF32 MMAs into one of two TMEM
//      accumulators, warps 0-3 store the result over the tile (the tile's loads
//      have all completed by then).
// Waits are bounded as in k_update_tc.
// ---------------------------------------------------------------------------
namespace {
constexpr uint32_t kTsBhi = 0;                        // B hi: 4 chunks [t][32 k], 128-byte swizzle
constexpr uint32_t kTsBlo = 4 * kOpBytes;             // B lo
constexpr uint32_t kTsA = 8 * kOpBytes;               // A stages: raw -> hi in place, lo
constexpr uint32_t kTsStage = 2 * kOpBytes;
constexpr int kTsStages = 3;
constexpr uint32_t kTsBar = kTsA + kTsStages * kTsStage;
constexpr uint32_t kTsSmem = kTsBar + 1024 + 1024;    // barriers, then alignment slack
constexpr int kTsLdW = 132;                           // column stride of the staged triangle
}  // namespace

__global__ void __launch_bounds__(kThreadsTc, 1)
    k_trsm_tc(SolveArgs a, const __grid_constant__ CUtensorMap tmap,
              const __grid_constant__ CUtensorMap tmap32, int K, long long spin) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  const Batch& bt = a.bt;
  const int b = bt.order[blockIdx.x];
  const int n = airfoil_n(bt, b), m = n + 1;
  if (!(m > kLargeM && n <= bt.n_max && a.info[b] == 0)) return;
  TlGeom g;
  g.init(m, bt.mat_off[b]);
  if (K < 1 || K >= g.T - 1) return;
  const int ns = g.T - 1 - K;
  const int kind = blockIdx.y & 1;  // 0: U12 tiles, 1: L21 tiles
  const int gy = (int)gridDim.y >> 1, y0 = (int)blockIdx.y >> 1;
  if (y0 >= ns) return;
  const int my_tiles = (ns - y0 + gy - 1) / gy;
  constexpr int nkc = kTlB / kKC;  // 4
  const int nq = my_tiles * nkc;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sraw = smem_u32(smraw);
  const uint32_t sbase = (sraw + 1023u) & ~1023u;
  unsigned char* gbase = smraw + (sbase - sraw);
  const uint32_t bar_base = sbase + kTsBar;
  // full[2] conv[2] empty[2] tfull[2] tempty[2] done
  auto full_bar = [&](int st) { return bar_base + 8u * st; };
  auto conv_bar = [&](int st) { return bar_base + 8u * (kTsStages + st); };
  auto empty_bar = [&](int st) { return bar_base + 8u * (2 * kTsStages + st); };
  auto tfull_bar = [&](int ac) { return bar_base + 8u * (3 * kTsStages + ac); };
  auto tempty_bar = [&](int ac) { return bar_base + 8u * (3 * kTsStages + 2 + ac); };
  const uint32_t done_bar = bar_base + 8u * (3 * kTsStages + 4);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(gbase + kTsBar + 128);
  volatile int* fail = reinterpret_cast<volatile int*>(gbase + kTsBar + 132);
  float* F = a.LU + bt.mat_off[b];

  // ---- 1. the inverse, as the B operand ----
  // Both solves need the inverse X of a lower triangular matrix W: W = L11
  // (unit diagonal) for U12, W = U11^T for L21 (then X = (U11^{-1})^T).  W is
  // staged column-major (WT[c][r] = W[r][c], columns 16-byte aligned, so a
  // piece of a column is a broadcast vector load) and inverted by 32 x 32
  // blocks: the four diagonal blocks X_ii = W_ii^{-1} are stored inverted in
  // the tile already, then the blocks at distance d = 1, 2, 3 below the
  // diagonal, X_ij = -X_ii sum_{j<=k<i} W_ik X_kj (all threads, 8 rows of one
  // column of a block each; W_ik, i > k, are the tile's untouched entries).
  {
    float* WT = reinterpret_cast<float*>(gbase + kTsA);       // 128 x kTsLdW, column-major
    float* X = reinterpret_cast<float*>(gbase);               // 128 x 128, row-major
    float* XD = reinterpret_cast<float*>(gbase + kTsBlo);     // 4 x 32 x 32, X_ii column-major
    const float* Td = F + g.tile(K, K);
    const bool unit = (kind == 0);
    // the tile's 16384 values, 26 loads of a thread in flight at a time
    constexpr int kPerT = (kTlTile + kThreadsTc - 1) / kThreadsTc;  // 52
    constexpr int kBatch = kPerT / 2;
    static_assert(2 * kBatch == kPerT, "two batches");
#pragma unroll 1
    for (int e0 = 0; e0 < kPerT; e0 += kBatch) {
      float v[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int e = tid + (e0 + u) * kThreadsTc, r = e >> 7, c = e & 127;
        v[u] = (e < kTlTile) ? __ldg(Td + ((c >> 5) << 12) + r * 32 + (c & 31)) : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int e = tid + (e0 + u) * kThreadsTc, r = e >> 7, c = e & 127;
        // kind 0: W = L (W[r][c] = tile(r, c)); kind 1: W = U^T (W[c][r] = tile(r, c))
        if (e < kTlTile) {
          if (kind == 0)
            WT[c * kTsLdW + r] = v[u];
          else
            WT[r * kTsLdW + c] = v[u];
        }
      }
    }
    __syncthreads();
    if (warp < 4) {
      // X_ii, i = warp, column `lane`: the diagonal tile's 32 x 32 diagonal
      // blocks hold L_ii^{-1} below the diagonal (unit diagonal implied) and
      // U_ii^{-1} on and above it (k_large_diag), so X_ii[t][l] = W_ii^{-1}[t][l]
      // is the staged WT value at (t, l) for t > l -- L_ii^{-1}[t][l], or for
      // W = U^T, U_ii^{-1}[l][t] -- and on the diagonal 1 (L) or U_ii^{-1}[l][l].
      const int i0 = 32 * warp;
#pragma unroll 4
      for (int t = 0; t < 32; ++t) {
        float v = 0.0f;
        if (t > lane || (t == lane && !unit)) v = WT[(i0 + lane) * kTsLdW + i0 + t];
        if (t == lane && unit) v = 1.0f;
        X[(i0 + t) * 128 + i0 + lane] = v;
        XD[warp * 1024 + lane * 32 + t] = v;  // column lane of X_ii
      }
    }
    // the strictly lower blocks are zero above the diagonal blocks
    for (int e = tid; e < kTlTile; e += kThreadsTc) {
      const int r = e >> 7, c = e & 127;
      if ((c >> 5) > (r >> 5)) X[e] = 0.0f;
    }
    __syncthreads();
    // The blocks at distance d = 1, 2, 3 below the diagonal, all threads: a
    // task is 8 rows x 1 column of a block (lane = column, so that the W and
    // X_ii values of the task's rows are broadcast vector loads).  First
    // T_ij = sum_{j<=k<i} W_ik X_kj into TB, then X_ij = -X_ii T_ij into X.
    float* TB = XD + 4 * 1024;  // 3 x 32 x 32, row-major per block
    for (int d = 1; d < 4; ++d) {
      const int ntask = (4 - d) * 128;
      for (int task = tid; task < ntask; task += kThreadsTc) {
        const int j = task >> 7, r0 = 8 * ((task >> 5) & 3), c = task & 31, i = j + d;
        float acc[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) acc[t] = 0.0f;
        for (int kk = 32 * j; kk < 32 * i; ++kk) {
          const float xv = X[kk * 128 + 32 * j + c];
          const float4 w0 = *reinterpret_cast<const float4*>(WT + kk * kTsLdW + 32 * i + r0);
          const float4 w1 = *reinterpret_cast<const float4*>(WT + kk * kTsLdW + 32 * i + r0 + 4);
          acc[0] = fmaf(w0.x, xv, acc[0]);
          acc[1] = fmaf(w0.y, xv, acc[1]);
          acc[2] = fmaf(w0.z, xv, acc[2]);
          acc[3] = fmaf(w0.w, xv, acc[3]);
          acc[4] = fmaf(w1.x, xv, acc[4]);
          acc[5] = fmaf(w1.y, xv, acc[5]);
          acc[6] = fmaf(w1.z, xv, acc[6]);
          acc[7] = fmaf(w1.w, xv, acc[7]);
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) TB[j * 1024 + (r0 + t) * 32 + c] = acc[t];
      }
      __syncthreads();
      for (int task = tid; task < ntask; task += kThreadsTc) {
        const int j = task >> 7, r0 = 8 * ((task >> 5) & 3), c = task & 31, i = j + d;
        const float* xd = XD + i * 1024;  // X_ii column-major: X_ii[t][kk] = xd[32 kk + t]
        float acc[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) acc[t] = 0.0f;
#pragma unroll 4
        for (int kk = 0; kk < 32; ++kk) {
          const float tv = TB[j * 1024 + kk * 32 + c];
          const float4 x0 = *reinterpret_cast<const float4*>(xd + kk * 32 + r0);
          const float4 x1 = *reinterpret_cast<const float4*>(xd + kk * 32 + r0 + 4);
          acc[0] = fmaf(-x0.x, tv, acc[0]);
          acc[1] = fmaf(-x0.y, tv, acc[1]);
          acc[2] = fmaf(-x0.z, tv, acc[2]);
          acc[3] = fmaf(-x0.w, tv, acc[3]);
          acc[4] = fmaf(-x1.x, tv, acc[4]);
          acc[5] = fmaf(-x1.y, tv, acc[5]);
          acc[6] = fmaf(-x1.z, tv, acc[6]);
          acc[7] = fmaf(-x1.w, tv, acc[7]);
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) X[(32 * i + r0 + t) * 128 + 32 * j + c] = acc[t];
      }
      __syncthreads();
    }
    // X -> the A region (W is no longer needed), then the B operand from it:
    // U12^T = A12^T (L11^{-1})^T needs B[t][k] = L11^{-1}[t][k] = X[t][k];
    // L21 = A21 U11^{-1} needs B[t][k] = U11^{-1}[k][t] = X[t][k] as well
    float* Xc = WT;
    for (int e = tid; e < kTlTile; e += kThreadsTc) Xc[e] = X[e];
    __syncthreads();
    for (int e = tid; e < kTlTile; e += kThreadsTc) {
      const int t = e >> 7, k = e & 127;  // along rows of X: conflict-free reads and writes
      const float v = Xc[t * 128 + k];
      const float h = tf32_hi(v);
      const uint32_t o = (uint32_t)(k >> 5) * kOpBytes + sw_off(t, k & 31);
      *reinterpret_cast<float*>(gbase + kTsBhi + o) = h;
      *reinterpret_cast<float*>(gbase + kTsBlo + o) = v - h;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int st = 0; st < kTsStages; ++st) {
      mbar_init(full_bar(st), 1);
      mbar_init(conv_bar(st), 4);
      mbar_init(empty_bar(st), 1);
    }
    for (int ac = 0; ac < 2; ++ac) {
      mbar_init(tfull_bar(ac), 1);
      mbar_init(tempty_bar(ac), 4);
    }
    mbar_init(done_bar, 1);
    *fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  // the task's tile: (K, J) of A12 (kind 0) or (I, K) of A21 (kind 1)
  auto tile_of = [&](int tau) {
    const int j = y0 + tau * gy;
    return (kind == 0) ? g.tile(K, K + 1 + j) : g.tile(K + 1 + j, K);
  };
  auto row_of = [&](int64_t tile_off, int kc) {
    return (int)((g.base + tile_off + (int64_t)kc * kTlChunk) >> 5);
  };

  if (warp == kWarpTma) {
    if (lane == 0) {
      int issued = 0;
      for (int q = 0; q < nq; ++q) {
        const int st = q % kTsStages, u = q / kTsStages;
        if (u >= 1 && !mbar_wait(empty_bar(st), (u - 1) & 1, fail, spin)) break;
        const int64_t t0 = tile_of(q / nkc);
        const int kk = q % nkc;
        const uint32_t raw = sbase + kTsA + st * kTsStage;
        mbar_arrive_tx(full_bar(st), kOpBytes);
        if (kind == 1) {
          tma_load(raw, &tmap, row_of(t0, kk), full_bar(st));
        } else {
          // rows k in [32 kk, 32 kk + 32) of each 32-column chunk of A12
#pragma unroll
          for (int c4 = 0; c4 < 4; ++c4)
            tma_load(raw + c4 * (kOpBytes / 4), &tmap32, row_of(t0, c4) + kKC * kk, full_bar(st));
        }
        issued = q + 1;
      }
      for (int q = max(0, issued - kTsStages); q < issued; ++q)
        mbar_wait_done(full_bar(q % kTsStages), (q / kTsStages) & 1);
    }
    __syncwarp();
  } else if (warp >= 4 && warp < 8) {
    const int ct = tid - 128;
    for (int q = 0; q < nq; ++q) {
      const int st = q % kTsStages, u = q / kTsStages;
      const bool ok = mbar_wait(full_bar(st), u & 1, fail, spin);
      if (!__all_sync(0xffffffffu, ok)) break;
      unsigned char* S = gbase + kTsA + st * kTsStage;  // raw -> hi, lo
      if (kind == 1) {
        // raw is already in the MMA's swizzled layout: split element by element
        float4* H4 = reinterpret_cast<float4*>(S);
        float4* L4 = reinterpret_cast<float4*>(S + kOpBytes);
#pragma unroll 4
        for (int j = 0; j < (int)(kOpBytes / 16) / 128; ++j) {
          const int i = ct + 128 * j;
          const float4 v = H4[i];
          const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
          H4[i] = h;
          L4[i] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
        }
      } else {
        // raw [c / 32][k][c % 32]: box w = ct / 32 holds columns c = 32 w .. of
        // A12, i.e. rows c of A^T, whose swizzled image (rows 32 w .. 32 w + 31,
        // 128 bytes each) is the same 4 KB: the warp reads its box into
        // registers (lane = c % 32, conflict-free) and writes it back transposed
        const int w = ct >> 5, c = 32 * w + lane;
        const float* R = reinterpret_cast<const float*>(S) + w * (kTM * kKC / 4);
        float col[kKC];
#pragma unroll
        for (int k = 0; k < kKC; ++k) col[k] = R[k * 32 + lane];
        __syncwarp();
#pragma unroll
        for (int j = 0; j < kKC / 4; ++j) {
          const uint32_t o = (uint32_t)(c * 128 + (((j ^ (c & 7)) & 7) << 4));
          const float4 h = make_float4(tf32_hi(col[4 * j]), tf32_hi(col[4 * j + 1]),
                                       tf32_hi(col[4 * j + 2]), tf32_hi(col[4 * j + 3]));
          *reinterpret_cast<float4*>(S + o) = h;
          *reinterpret_cast<float4*>(S + kOpBytes + o) =
              make_float4(col[4 * j] - h.x, col[4 * j + 1] - h.y, col[4 * j + 2] - h.z,
                          col[4 * j + 3] - h.w);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(conv_bar(st));
    }
  } else if (warp == kWarpMma) {
    if (lane == 0) {
      for (int q = 0; q < nq; ++q) {
        const int st = q % kTsStages, u = q / kTsStages;
        const int kk = q % nkc, tau = q / nkc, ac = tau & 1, v = tau >> 1;
        if (kk == 0 && v >= 1 && !mbar_wait(tempty_bar(ac), (v - 1) & 1, fail, spin)) break;
        if (!mbar_wait(conv_bar(st), u & 1, fail, spin)) break;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(ac * kTN);
        const uint32_t ah = sbase + kTsA + st * kTsStage, al = ah + kOpBytes;
        const uint32_t bh = sbase + kTsBhi + kk * kOpBytes, bl = sbase + kTsBlo + kk * kOpBytes;
#pragma unroll
        for (int s = 0; s < kKC / 8; ++s) {
          const uint32_t ko = 32u * s;
          const uint32_t acc0 = (kk > 0 || s > 0) ? 1u : 0u;
          tc_mma(d, desc_sw128(ah + ko), desc_sw128(bh + ko), acc0);
          tc_mma(d, desc_sw128(ah + ko), desc_sw128(bl + ko), 1u);
          tc_mma(d, desc_sw128(al + ko), desc_sw128(bh + ko), 1u);
        }
        tc_commit(empty_bar(st));
        if (kk == nkc - 1) tc_commit(tfull_bar(ac));
      }
      tc_commit(done_bar);
    }
    __syncwarp();
  } else {
    // ---- epilogue: D over the tile (U12 transposed): row = M index ----
    const int r = 32 * warp + lane;
    for (int tau = 0; tau < my_tiles; ++tau) {
      const int ac = tau & 1, v = tau >> 1;
      if (!epi_all(mbar_wait(tfull_bar(ac), v & 1, fail, spin))) break;
      tc_fence_after();
      float* out = F + tile_of(tau);
#pragma unroll 1
      for (int s = 0; s < kTN / kKC; ++s) {
        float v32[32];
        tc_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(ac * kTN + kKC * s), v32);
        if (s == kTN / kKC - 1) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(tempty_bar(ac));
        }
        float4* o4 = reinterpret_cast<float4*>(out + (int64_t)s * kTlChunk + r * 32);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          o4[j] = make_float4(v32[4 * j], v32[4 * j + 1], v32[4 * j + 2], v32[4 * j + 3]);
      }
    }
  }

  __syncthreads();
  const bool drained = mbar_wait_done(done_bar, 0);
  if (!drained || *fail) {
    if (tid == 0) a.info[b] = PANEL_INFO_DEVICE_TIMEOUT;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
}

// The tensor map of the factor buffer as rows of 32 floats (128 bytes), boxes
// of 128 rows (one chunk), 128-byte swizzle.  `floats` bounds the buffer's
// size from above; only chunks inside the caller's buffer are ever addressed.
static cudaError_t encode_map(float* base, uint64_t floats, uint32_t box_rows, bool swizzle,
                              CUtensorMap* out);

cudaError_t make_update_map(float* base, uint64_t floats, UpdateMap* out) {
  cudaError_t e = encode_map(base, floats, kTM, true, &out->map);
  if (e == cudaSuccess) e = encode_map(base, floats, kKC, false, &out->map32);
  return e;
}

// rows of 32 floats, boxes of `box_rows` rows; 128-byte swizzle or none
static cudaError_t encode_map(float* base, uint64_t floats, uint32_t box_rows, bool swizzle,
                              CUtensorMap* out) {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                         cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  if (!encode) return cudaErrorNotSupported;
  if ((reinterpret_cast<uintptr_t>(base) & 15u) != 0) return cudaErrorMisalignedAddress;
  uint64_t rows = (floats + kTlC - 1) / kTlC;
  if (rows > 0xFFFFFFFFull) rows = 0xFFFFFFFFull;
  if (rows < (uint64_t)kTM) rows = kTM;
  const cuuint64_t dims[2] = {(cuuint64_t)kTlC, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)kTlC * 4};
  const cuuint32_t box[2] = {(cuuint32_t)kTlC, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE,
                            swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t ensure_update_smem() {
  const cudaError_t e = ensure_smem(k_update_tc, (size_t)kSmemBytes);
  return e != cudaSuccess ? e : ensure_smem(k_trsm_tc, (size_t)kTsSmem);
}

cudaError_t launch_trsm_tc(const SolveArgs& a, const UpdateMap& map, int K, int split,
                           long long spin, cudaStream_t s) {
  k_trsm_tc<<<dim3(a.bt.B, 2 * split), kThreadsTc, kTsSmem, s>>>(a, map.map, map.map32, K, spin);
  return cudaGetLastError();
}

cudaError_t launch_update_tc(const SolveArgs& a, const UpdateMap& map, int K, int split,
                             long long spin, cudaStream_t s) {
  k_update_tc<<<dim3(a.bt.B, split), kThreadsTc, kSmemBytes, s>>>(a, map.map, K, spin);
  return cudaGetLastError();
}

}  // namespace panel
