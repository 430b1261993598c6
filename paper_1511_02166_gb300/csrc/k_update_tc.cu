// k_update_tc.cu -- the trailing update A22 -= L21 U12 of the step-synchronous
// blocked LU of large airfoils (k_lu_large.cu) on the 5th-generation tensor
// cores: tcgen05.mma (kind::tf32) with the accumulator in tensor memory.
//
// One block takes 128 x 128 output tiles of one airfoil (block y of gridDim.y
// strides over the airfoil's tiles); K = 128 (the block column) is fed in
// chunks of kKC = 16.  The block is warp-specialised (288 threads):
//   warps 0-3  epilogue: wait for a finished accumulator, read it from tensor
//              memory (warp w owns TMEM lanes 32w..32w+31 = tile rows) and
//              subtract it from A22;
//   warps 4-7  producers: load a chunk of L21 and U12 into registers (the
//              next chunk is in flight while the current one is stored), split
//              it into TF32 hi / lo parts and store them in shared memory;
//   warp 8     one lane issues the MMAs.
// Producers and the MMA lane pass kStages shared-memory stages through
// full / empty mbarriers; the MMA lane and the epilogue pass two tensor-memory
// accumulators (2 x 128 columns) through tfull / tempty mbarriers, so the
// epilogue of one tile overlaps the MMAs of the next.
//
// Precision.  The factor is FP32; a TF32 product alone (11 significant bits)
// would make the LU far less accurate than FP32 and the refinement would stall
// on these ill-conditioned systems.  Each operand is split x = x_hi + x_lo with
// x_hi = x rounded to TF32 and x_lo = x - x_hi (exact in FP32), and the
// product is formed as A_hi B_hi + A_hi B_lo + A_lo B_hi (three MMAs per K
// step, the dropped A_lo B_lo is ~2^-22 relative), accumulated in FP32 in
// tensor memory.  The rank-128 product is accumulated on its own and
// subtracted from A22 once, in the epilogue.
//
// Layout.  The airfoil's row stride m is arbitrary, so rows are not 16-byte
// aligned and a tensor map cannot describe them; the producers write the
// canonical K-major, non-swizzled layout themselves: 8-row x 16-byte core
// matrices, 128 contiguous bytes each; core matrices adjacent in K are 128 B
// apart (leading byte offset), those adjacent in M / N are kKC / 4 x 128 B
// apart (stride byte offset).  A generic-to-async proxy fence orders the
// stores before the MMAs that read them.
//
// Every pipeline wait is bounded (`spin` polls, a kernel argument) and polls a
// shared failure flag: a block that gives up stops issuing work, and every
// role leaves its loop.  The MMA lane commits a final arrival on done_bar on
// every path, after the last MMA it issued; the block then waits for that
// arrival with its own bound (kDoneLimit, independent of `spin` and of the
// failure flag), so that no MMA is still reading shared memory or writing
// tensor memory when the block sets info[b] = PANEL_INFO_DEVICE_TIMEOUT, frees
// its tensor memory and returns.
#include "lu_mixed.cuh"

namespace panel {

namespace {

constexpr int kTM = 128;               // tile rows (MMA M)
constexpr int kTN = 128;               // tile columns (MMA N)
constexpr int kKC = 16;                // K per chunk
constexpr int kBWc = 128;              // block column width (K of the update)
constexpr int kChunks = kBWc / kKC;    // 8
constexpr int kStages = 3;             // shared-memory stages
constexpr int kOpBytes = kTM * kKC * 4;            // one operand plane of a chunk: 8 KB
constexpr int kBufBytes = 4 * kOpBytes;            // A_hi, A_lo, B_hi, B_lo
constexpr int kSmemBytes = kStages * kBufBytes + 128;  // stages + barriers + flags
constexpr uint32_t kTmemCols = 2 * kTN;            // two FP32 accumulators, 128 x 128 each
constexpr int kThreadsTc = 288;                    // 4 epilogue + 4 producer + 1 MMA warps
// bound of the final wait for the block's own MMAs (they finish in
// microseconds; the bound only keeps the wait finite)
constexpr long long kDoneLimit = 1ll << 24;

// Instruction descriptor, kind::tf32: D = F32 (bits 4-5 = 1), A = B = TF32
// (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22,
// M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);

// Shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading
// byte offset >> 4 (16-29), stride byte offset >> 4 (32-45), descriptor
// version 1 (bit 46), no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  constexpr uint64_t lbo = 128 >> 4;
  constexpr uint64_t sbo = ((kKC / 4) * 128) >> 4;
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | (lbo << 16) | (sbo << 32) | (1ull << 46);
}

// Byte offset of element (row, k) of a kTM x kKC operand plane in the
// canonical layout.
__device__ __forceinline__ uint32_t core_off(int row, int k) {
  return (uint32_t)((((row >> 3) * (kKC / 4) + (k >> 2)) << 7) + ((row & 7) << 4) + ((k & 3) << 2));
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

// The final wait for the block's own MMAs: bounded, but it does not give up
// when *fail is set (the MMAs issued before the failure are still running).
__device__ __forceinline__ bool mbar_wait_done(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < kDoneLimit; ++it)
    if (mbar_try(bar, parity)) return true;
  return false;
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

__global__ void __launch_bounds__(kThreadsTc, 2) k_update_tc(SolveArgs a, int k0,
                                                              long long spin) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  const Batch& bt = a.bt;
  const int b = bt.order[blockIdx.x];
  const int n = airfoil_n(bt, b), m = n + 1;
  if (!(m > kLargeM && n <= bt.n_max && a.info[b] == 0)) return;
  const int k1 = k0 + kBWc;
  if (k1 >= m) return;
  const int rest = m - k1, nt = (rest + kTN - 1) / kTN, tiles = nt * nt;
  if ((int)blockIdx.y >= tiles) return;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float* F = a.LU + bt.mat_off[b];
  unsigned char* misc = smraw + kStages * kBufBytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(misc);  // full[3] empty[3] tfull[2] tempty[2] done
  uint32_t* tslot = reinterpret_cast<uint32_t*>(misc + 96);
  volatile int* fail = reinterpret_cast<volatile int*>(misc + 100);
  const uint32_t sbase = smem_u32(smraw);
  const uint32_t bar_base = smem_u32(bars);
  auto full_bar = [&](int st) { return bar_base + 8u * st; };
  auto empty_bar = [&](int st) { return bar_base + 8u * (kStages + st); };
  auto tfull_bar = [&](int ac) { return bar_base + 8u * (2 * kStages + ac); };
  auto tempty_bar = [&](int ac) { return bar_base + 8u * (2 * kStages + 2 + ac); };
  const uint32_t done_bar = bar_base + 8u * (2 * kStages + 4);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int st = 0; st < kStages; ++st) {
      mbar_init(full_bar(st), 4);   // one arrival per producer warp
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

  const int my_tiles = (tiles - (int)blockIdx.y + (int)gridDim.y - 1) / (int)gridDim.y;
  const int nq = my_tiles * kChunks;
  auto tile_rc = [&](int tau, int& r0, int& c0) {
    const int t = (int)blockIdx.y + tau * (int)gridDim.y;
    r0 = k1 + (t / nt) * kTM;
    c0 = k1 + (t % nt) * kTN;
  };

  if (warp >= 4 && warp < 8) {
    // ---------------- producers ----------------
    const int pt = tid - 128;
    constexpr int kPer = kTM * kKC / 128;  // 16 values of A and 16 of B^T per thread
    auto load = [&](int q, float (&ra)[kPer], float (&rb)[kPer]) {
      int r0, c0;
      tile_rc(q / kChunks, r0, c0);
      const int kg = k0 + (q % kChunks) * kKC;
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        const int e = pt + 128 * j;
        const int r = r0 + (e >> 4);          // A[row][k], k fastest
        ra[j] = (r < m) ? F[r * m + kg + (e & 15)] : 0.0f;
        const int c = c0 + (e & 127);         // U12[k][col], col fastest
        rb[j] = (c < m) ? F[(kg + (e >> 7)) * m + c] : 0.0f;
      }
    };
    auto store = [&](int q, const float (&ra)[kPer], const float (&rb)[kPer]) -> bool {
      const int st = q % kStages, u = q / kStages;
      if (u >= 1 && !mbar_wait(empty_bar(st), (u - 1) & 1, fail, spin)) return false;
      unsigned char* B = smraw + st * kBufBytes;
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        const int e = pt + 128 * j;
        const uint32_t oa = core_off(e >> 4, e & 15);
        const float ha = tf32_hi(ra[j]);
        *reinterpret_cast<float*>(B + oa) = ha;
        *reinterpret_cast<float*>(B + kOpBytes + oa) = ra[j] - ha;
        const uint32_t ob = core_off(e & 127, e >> 7);
        const float hb = tf32_hi(rb[j]);
        *reinterpret_cast<float*>(B + 2 * kOpBytes + ob) = hb;
        *reinterpret_cast<float*>(B + 3 * kOpBytes + ob) = rb[j] - hb;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(full_bar(st));
      return true;
    };
    float a0[kPer], b0[kPer], a1[kPer], b1[kPer];
    load(0, a0, b0);
    for (int q = 0; q < nq; q += 2) {
      if (q + 1 < nq) load(q + 1, a1, b1);
      if (!store(q, a0, b0)) break;
      if (q + 1 >= nq) break;
      if (q + 2 < nq) load(q + 2, a0, b0);
      if (!store(q + 1, a1, b1)) break;
    }
  } else if (warp == 8) {
    // ---------------- MMA issue (one lane) ----------------
    if (lane == 0) {
      for (int q = 0; q < nq; ++q) {
        const int st = q % kStages, u = q / kStages;
        const int kc = q % kChunks, tau = q / kChunks, ac = tau & 1, v = tau >> 1;
        if (kc == 0 && v >= 1 && !mbar_wait(tempty_bar(ac), (v - 1) & 1, fail, spin)) break;
        if (!mbar_wait(full_bar(st), u & 1, fail, spin)) break;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(ac * kTN);
        const uint32_t ah = sbase + st * kBufBytes, al = ah + kOpBytes;
        const uint32_t bh = ah + 2 * kOpBytes, bl = ah + 3 * kOpBytes;
#pragma unroll
        for (int s = 0; s < kKC / 8; ++s) {  // K = 8 per MMA: two core matrices
          const uint32_t ko = s * 2 * 128;
          const uint32_t acc0 = (kc > 0 || s > 0) ? 1u : 0u;
          tc_mma(d, smem_desc(ah + ko), smem_desc(bh + ko), acc0);
          tc_mma(d, smem_desc(ah + ko), smem_desc(bl + ko), 1u);
          tc_mma(d, smem_desc(al + ko), smem_desc(bh + ko), 1u);
        }
        tc_commit(empty_bar(st));
        if (kc == kChunks - 1) tc_commit(tfull_bar(ac));
      }
      tc_commit(done_bar);  // arrives once every MMA issued above has completed
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: A22 -= D ----------------
    for (int tau = 0; tau < my_tiles; ++tau) {
      const int ac = tau & 1, v = tau >> 1;
      if (!mbar_wait(tfull_bar(ac), v & 1, fail, spin)) break;
      tc_fence_after();
      int r0, c0;
      tile_rc(tau, r0, c0);
      const int r = r0 + 32 * warp + lane;
#pragma unroll 1
      for (int s = 0; s < kTN / 32; ++s) {
        float v32[32];
        tc_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(ac * kTN + 32 * s), v32);
        if (r < m) {
          float* row = F + r * m + c0 + 32 * s;
          const int cn = min(32, m - (c0 + 32 * s));
          float c[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) c[i] = (i < cn) ? row[i] : 0.0f;
#pragma unroll
          for (int i = 0; i < 32; ++i)
            if (i < cn) row[i] = c[i] - v32[i];
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty_bar(ac));
    }
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

size_t update_tc_smem() { return (size_t)kSmemBytes; }

}  // namespace panel
