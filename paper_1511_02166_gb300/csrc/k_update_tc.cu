// k_update_tc.cu -- the trailing update A22 -= L21 U12 of the step-synchronous
// blocked LU of large airfoils (k_lu_large.cu) on the 5th-generation tensor
// cores: tcgen05.mma (kind::tf32) with the accumulator in tensor memory.
//
// One block of 256 threads takes 128 x 128 output tiles of one airfoil (block
// y of gridDim.y strides over the airfoil's tiles); K = 128 (the block column)
// in chunks of kKC = 16, double-buffered in shared memory.
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
// Data movement.  The airfoil's row stride m is arbitrary, so rows are not
// 16-byte aligned and a tensor map cannot describe them: operand chunks are
// copied by cp.async (4 bytes per copy, zero-filled outside the matrix) into a
// ring of raw stages two chunks ahead, then split into hi / lo and written in
// the canonical K-major, non-swizzled layout:
// 8-row x 16-byte core matrices, 128 contiguous bytes each; core matrices
// adjacent in K are 128 B apart (leading byte offset), those adjacent in M / N
// are kKC / 4 x 128 B apart (stride byte offset).  A generic-to-async proxy
// fence orders the stores before the MMAs that read them; tcgen05.commit
// arrives on one mbarrier per buffer when the MMAs that read it are done.
// The epilogue reads the accumulator with tcgen05.ld (warp w reads TMEM lanes
// 32 (w % 4) .. + 31, i.e. rows of the tile, and columns 64 (w / 4) .. + 63).
//
// Every wait is bounded: a block that gives up sets info[b] =
// PANEL_INFO_DEVICE_TIMEOUT, stops issuing work, waits (bounded) for its own
// MMAs, frees its tensor memory and returns.
#include "lu_mixed.cuh"

namespace panel {

namespace {

constexpr int kTM = 128;               // tile rows (MMA M)
constexpr int kTN = 128;               // tile columns (MMA N)
constexpr int kKC = 16;                // K per staged chunk
constexpr int kBWc = 128;              // block column width (K of the update)
constexpr int kChunks = kBWc / kKC;    // 8
constexpr int kOpBytes = kTM * kKC * 4;            // one operand plane of a chunk: 8 KB
constexpr int kBufBytes = 4 * kOpBytes;            // A_hi, A_lo, B_hi, B_lo
constexpr int kRawStages = 3;                      // raw chunks in flight (cp.async)
constexpr int kRawBytes = 2 * kOpBytes;            // raw A and B^T of one chunk
constexpr int kSmemBytes = 2 * kBufBytes + kRawStages * kRawBytes + 64;
constexpr uint32_t kTmemCols = 128;                // FP32 accumulator, 128 x 128
constexpr long long kSpinLimit = 1ll << 22;        // bounded waits (well under a second per wait)

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

// Waits for the phase with the given parity; false if the bounded spin ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
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

__global__ void __launch_bounds__(256, 2) k_update_tc(SolveArgs a, int k0) {
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
  unsigned char* raw = smraw + 2 * kBufBytes;  // kRawStages x (A rows, B^T rows)
  unsigned char* misc = raw + kRawStages * kRawBytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(misc);  // 2 barriers
  uint32_t* tslot = reinterpret_cast<uint32_t*>(misc + 16);
  int* fail = reinterpret_cast<int*>(misc + 20);
  const uint32_t sbase = smem_u32(smraw);
  const uint32_t rbase = smem_u32(raw);
  const uint32_t bar0 = smem_u32(&bars[0]), bar1 = smem_u32(&bars[1]);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar1, 1);
    *fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  uint32_t phase[2] = {0u, 0u};
  bool pending[2] = {false, false};
  bool ok = true;

  // The chunks of all this block's tiles form one sequence q = 0 .. nq - 1
  // (kChunks per tile).  Raw copies (cp.async, 4 bytes each: rows are not
  // 16-byte aligned) run kRawStages - 1 chunks ahead of the MMAs.
  const int my_tiles = (tiles - (int)blockIdx.y + (int)gridDim.y - 1) / (int)gridDim.y;
  const int nq = my_tiles * kChunks;
  constexpr int kPer = kTM * kKC / 256;  // elements of A (and of B^T) per thread per chunk
  auto tile_of = [&](int q, int& r0, int& c0) {
    const int t = (int)blockIdx.y + (q / kChunks) * (int)gridDim.y;
    r0 = k1 + (t / nt) * kTM;
    c0 = k1 + (t % nt) * kTN;
  };
  auto issue = [&](int q) {
    if (q < nq) {
      int r0, c0;
      tile_of(q, r0, c0);
      const int kg = k0 + (q % kChunks) * kKC;
      const uint32_t dst = rbase + (uint32_t)((q % kRawStages) * kRawBytes);
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        const int e = tid + 256 * j;
        const int r = r0 + e / kKC;                    // A[row][k], k fastest
        const bool va = r < m;
        const float* sa = va ? F + r * m + kg + e % kKC : F;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst + 4 * e), "l"(sa),
                     "r"(va ? 4 : 0)
                     : "memory");
        const int c = c0 + e % kTN;                    // B^T raw as U12[k][col], col fastest
        const bool vb = c < m;
        const float* sb = vb ? F + (kg + e / kTN) * m + c : F;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst + kOpBytes + 4 * e),
                     "l"(sb), "r"(vb ? 4 : 0)
                     : "memory");
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  for (int q = 0; q < kRawStages - 1; ++q) issue(q);
  for (int q = 0; q < nq && ok; ++q) {
    const int kc = q % kChunks, buf = q & 1;
    asm volatile("cp.async.wait_group %0;" ::"n"(kRawStages - 2) : "memory");
    __syncthreads();  // chunk q's raw copy is visible to every thread
    if (pending[buf]) {  // the MMAs that read this buffer two chunks ago
      if (!mbar_wait(buf ? bar1 : bar0, phase[buf])) *fail = 1;
      phase[buf] ^= 1u;
      pending[buf] = false;
    }
    {
      const float* ra = reinterpret_cast<const float*>(raw + (q % kRawStages) * kRawBytes);
      const float* rb = ra + kTM * kKC;
      unsigned char* B = smraw + buf * kBufBytes;
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        const int e = tid + 256 * j;
        const float xa = ra[e];
        const float ha = tf32_hi(xa);
        const uint32_t oa = core_off(e / kKC, e % kKC);
        *reinterpret_cast<float*>(B + oa) = ha;
        *reinterpret_cast<float*>(B + kOpBytes + oa) = xa - ha;
        const float xb = rb[e];
        const float hb = tf32_hi(xb);
        const uint32_t ob = core_off(e % kTN, e / kTN);
        *reinterpret_cast<float*>(B + 2 * kOpBytes + ob) = hb;
        *reinterpret_cast<float*>(B + 3 * kOpBytes + ob) = xb - hb;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (*fail) {
      ok = false;
      break;
    }
    if (tid == 0) {
      tc_fence_after();
      const uint32_t ah = sbase + buf * kBufBytes, al = ah + kOpBytes;
      const uint32_t bh = ah + 2 * kOpBytes, bl = ah + 3 * kOpBytes;
#pragma unroll
      for (int s = 0; s < kKC / 8; ++s) {  // K = 8 per MMA: two core matrices
        const uint32_t ko = s * 2 * 128;
        const uint32_t acc0 = (kc > 0 || s > 0) ? 1u : 0u;
        tc_mma(tmem, smem_desc(ah + ko), smem_desc(bh + ko), acc0);
        tc_mma(tmem, smem_desc(ah + ko), smem_desc(bl + ko), 1u);
        tc_mma(tmem, smem_desc(al + ko), smem_desc(bh + ko), 1u);
      }
      tc_commit(buf ? bar1 : bar0);
    }
    pending[buf] = true;
    issue(q + kRawStages - 1);
    if (kc != kChunks - 1) continue;

    // end of a tile: wait for all its MMAs, then A22 -= D
    for (int p = 0; p < 2; ++p) {
      if (pending[p]) {
        if (!mbar_wait(p ? bar1 : bar0, phase[p])) *fail = 1;
        phase[p] ^= 1u;
        pending[p] = false;
      }
    }
    tc_fence_after();
    __syncthreads();
    if (*fail) {
      ok = false;
      break;
    }
    int r0, c0;
    tile_of(q, r0, c0);
    const int g = warp & 3, h = warp >> 2;
    const int r = r0 + 32 * g + lane;
#pragma unroll 1
    for (int s = 0; s < 2; ++s) {
      const int cb = 64 * h + 32 * s;
      float v[32];
      tc_ld32(tmem + ((uint32_t)(32 * g) << 16) + (uint32_t)cb, v);
      if (r < m) {
        float* row = F + r * m + c0 + cb;
        const int cn = min(32, m - (c0 + cb));
        float c[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) c[i] = (i < cn) ? row[i] : 0.0f;
#pragma unroll
        for (int i = 0; i < 32; ++i)
          if (i < cn) row[i] = c[i] - v[i];
      }
    }
    tc_fence_before();
    __syncthreads();
  }

  asm volatile("cp.async.wait_all;" ::: "memory");
  if (!ok) {
    // give the MMAs already issued a bounded chance to finish before the
    // tensor memory is released
    if (tid == 0) a.info[b] = PANEL_INFO_DEVICE_TIMEOUT;
    for (int p = 0; p < 2; ++p)
      if (pending[p]) mbar_wait(p ? bar1 : bar0, phase[p]);
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
