// capi_noalloc.cu -- panel_solve_noalloc: panel_solve for callers that cannot
// allocate device memory.
//
// panel_solve needs two work arrays besides its inputs and outputs: the factor
// buffer (sum m_b^2 elements) and the pivots (sum m_b).  Some callers have no
// way to provide them: code that runs where cudaMalloc is not available or not
// allowed (a plug-in inside a host application that owns every allocation, a
// real-time loop that must not allocate after start-up, a foreign-language
// binding with no device allocator of its own).  For them this entry point
// keeps both arrays in one file-scope device array of fixed size, which the
// CUDA runtime sets aside when the library's device code is loaded on a GPU and
// holds until the process exits.  The caller still passes every input and
// output.  The kernels are those of panel_solve; only where the factor and the
// pivots live differs.
#include <mutex>

#include "panel_common.cuh"

namespace panel {
cudaError_t launch_solve_f64(const Batch&, const double*, double*, int32_t*, const double*,
                             const double*, const double*, double*, double*, int32_t*, int32_t*,
                             cudaStream_t);
cudaError_t launch_lu_mixed(const Batch&, const float*, float*, int32_t*, int32_t*, int32_t*,
                            bool, cudaStream_t, int lu_kind = 0);
cudaError_t launch_ir_mixed(const Batch&, const float*, const float*, const float*,
                            const int32_t*, const double*, const double*, const double*, double*,
                            double*, int, double, int32_t*, int32_t*, cudaStream_t,
                            int rhs_kind, int ir_shape);
}  // namespace panel

namespace {

// The factor and the pivots of the last call.  Nothing in it needs to start at
// zero: the factorisation writes every factor entry and pivot that the solves
// read.
static __device__ __align__(256) unsigned char g_solve_scratch[PANEL_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_solve_scratch on the current device, looked up once per
// device.  In host code the array's name only stands for the symbol; the
// address the kernels need comes from cudaGetSymbolAddress.
cudaError_t scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_solve_scratch);
    if (e != cudaSuccess) return e;
    if (!p) return cudaErrorInvalidSymbol;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

constexpr size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

extern "C" {

int panel_solve_noalloc(int B, int n_max, int flags, const int64_t* node_offsets_host,
                        const double* nodes, const int64_t* node_offsets,
                        const int64_t* mat_offsets, const int32_t* order, const double* A64,
                        const float* A_hi, const float* A_lo, const double* rhs,
                        const double* vinf, const double* chord, double* u, double* lambda,
                        int max_iter, double tol, int32_t* info, int32_t* iters, void* stream) {
  if (B < 0 || n_max < 3 || n_max > PANEL_N_MAX) return PANEL_EINVAL;
  const int mode = flags & (PANEL_FP64 | PANEL_MIXED);
  const bool adj = (flags & PANEL_WITH_ADJOINT) != 0;
  if ((mode != PANEL_FP64 && mode != PANEL_MIXED) ||
      (flags & ~(PANEL_FP64 | PANEL_MIXED | PANEL_WITH_ADJOINT | PANEL_INVERSE)) != 0 ||
      ((flags & PANEL_INVERSE) && mode != PANEL_MIXED))
    return PANEL_EINVAL;
  if (B == 0) return PANEL_OK;
  if (!node_offsets_host || !node_offsets || !mat_offsets || !order || !rhs || !u || !info)
    return PANEL_EINVAL;
  if (adj && (!lambda || !nodes)) return PANEL_EINVAL;
  if (mode == PANEL_FP64 && !A64) return PANEL_EINVAL;
  if (mode == PANEL_MIXED && (!A_hi || !A_lo || max_iter < 0 || !(tol > 0.0)))
    return PANEL_EINVAL;

  // the factor (sum m_b^2 elements) and, 256-byte aligned after it, the pivots
  // (sum m_b): both must fit the static array
  size_t mat = 0, vec = 0;
  for (int b = 0; b < B; ++b) {
    const int64_t n = node_offsets_host[b + 1] - node_offsets_host[b];
    if (n < 0) return PANEL_EINVAL;
    if (n > n_max) return PANEL_EINVAL;
    mat += (size_t)(n + 1) * (size_t)(n + 1);
    vec += (size_t)(n + 1);
  }
  const size_t esize = (mode == PANEL_FP64) ? sizeof(double) : sizeof(float);
  const size_t piv_off = round_up(mat * esize, 256);
  if (piv_off + vec * sizeof(int32_t) > (size_t)PANEL_NOALLOC_SCRATCH_BYTES)
    return PANEL_ESCRATCH;

  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return PANEL_ECUDA;
  void* LU = base;
  int32_t* piv = reinterpret_cast<int32_t*>(static_cast<unsigned char*>(base) + piv_off);

  panel::Batch bt;
  bt.B = B;
  bt.n_max = n_max;
  bt.nodes = nodes;
  bt.node_off = node_offsets;
  bt.mat_off = mat_offsets;
  bt.order = order;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (mode == PANEL_FP64) {
    e = panel::launch_solve_f64(bt, A64, static_cast<double*>(LU), piv, rhs, vinf, chord, u,
                                adj ? lambda : nullptr, info, iters, s);
  } else {
    e = panel::launch_lu_mixed(bt, A_hi, static_cast<float*>(LU), piv, info, iters,
                               (flags & PANEL_INVERSE) != 0, s);
    if (e == cudaSuccess)
      e = panel::launch_ir_mixed(bt, A_hi, A_lo, static_cast<const float*>(LU), piv, rhs, vinf,
                                 chord, u, adj ? lambda : nullptr, max_iter, tol, info, iters, s,
                                 0, 0);
  }
  return e == cudaSuccess ? PANEL_OK : PANEL_ECUDA;
}

}  // extern "C"
