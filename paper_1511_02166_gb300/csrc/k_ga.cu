// k_ga.cu -- the genetic algorithm around the batched evaluator (the genetic
// optimisation of Section 2): the B-spline genome sampled into panel nodes, and
// one generation of tournament selection, one-point crossover and mutation.
//
// Genome.  An airfoil is a clamped uniform cubic B-spline over P control
// points whose x coordinates are fixed for the whole population (ctrl_x, from
// the trailing edge over the upper surface to the leading edge and back over
// the lower surface); the genome is the P y coordinates.  Node i of n is the
// curve at parameter t_i, cosine-clustered towards both ends of each half of
// the parameter range (the trailing and the leading edge):
//   i <= n_u = ceil(n / 2):  t_i = (1 - cos(pi i / n_u)) / 4
//   i >  n_u:                t_i = 1/2 + (1 - cos(pi (i - n_u) / (n - n_u))) / 4.
// The basis functions are evaluated by the Cox-de Boor recursion (FP64).
//
// Generation step (one thread per pair of children; every random number is an
// input, uniform in [0, 1), R = 4k + 5 per pair in this order):
//   two tournaments, each: k candidate indices floor(u B) (with replacement),
//   ranked by fitness (higher first; NaN ranks last; ties by lower index, then
//   by draw order), then k - 1 acceptance draws: the j-th ranked candidate is
//   taken at the first draw below p (probability p (1-p)^j), the last one if
//   none is;
//   one-point crossover at c = 1 + floor(u (P - 1)) in [1, P-1]: child 1 takes
//   genes [0, c) from the first parent and [c, P) from the second, child 2 the
//   reverse;
//   per child, mutation: with probability pm gene floor(u P) moves by
//   sigma_g (2u - 1) and is clamped to [lo_g, hi_g].
#include "panel_common.cuh"

namespace panel {

namespace {

// Cubic basis functions N[0..3] of the knot span containing t; returns the
// span s (control points s-3 .. s carry N[0..3]).
__device__ __forceinline__ int bspline_basis3(double t, int P, double (&N)[4]) {
  const int segs = P - 3;
  int j = (int)floor(t * segs);
  if (j > segs - 1) j = segs - 1;
  if (j < 0) j = 0;
  const int s = j + 3;
  auto knot = [&](int q) -> double {
    if (q <= 3) return 0.0;
    if (q >= P) return 1.0;
    return (double)(q - 3) / segs;
  };
  double left[4], right[4];
  N[0] = 1.0;
  for (int d = 1; d <= 3; ++d) {
    left[d] = t - knot(s + 1 - d);
    right[d] = knot(s + d) - t;
    double saved = 0.0;
    for (int r = 0; r < d; ++r) {
      const double tmp = N[r] / (right[r + 1] + left[d - r]);
      N[r] = saved + right[r + 1] * tmp;
      saved = left[d - r] * tmp;
    }
    N[d] = saved;
  }
  return s;
}

__device__ __forceinline__ bool fitter(double fa, int ia, int pa, double fb, int ib, int pb) {
  // a ranks before b: higher fitness (NaN lowest), then lower index, then draw order
  const bool na = !(fa == fa), nb = !(fb == fb);
  if (na != nb) return nb;
  if (!na && fa != fb) return fa > fb;
  if (ia != ib) return ia < ib;
  return pa < pb;
}

constexpr int kMaxTournament = 16;

__device__ int tournament(int B, int k, double p, const double* __restrict__ fitness,
                          const double* __restrict__ u) {
  int idx[kMaxTournament], pos[kMaxTournament];
  for (int j = 0; j < k; ++j) {
    int c = (int)floor(__dmul_rn(u[j], (double)B));
    idx[j] = c < B ? c : B - 1;
    pos[j] = j;
  }
  // insertion sort of the k candidates by rank
  for (int a = 1; a < k; ++a) {
    const int ia = idx[a], pa = pos[a];
    int b = a - 1;
    while (b >= 0 && fitter(fitness[ia], ia, pa, fitness[idx[b]], idx[b], pos[b])) {
      idx[b + 1] = idx[b];
      pos[b + 1] = pos[b];
      --b;
    }
    idx[b + 1] = ia;
    pos[b + 1] = pa;
  }
  for (int j = 0; j < k - 1; ++j)
    if (u[k + j] < p) return idx[j];
  return idx[k - 1];
}

}  // namespace

// Nodes of a tile of kTileN nodes x kTileB airfoils per block: the basis of the
// tile's nodes (and their x, shared by the population) is evaluated once into
// shared memory, then every airfoil of the tile applies it to its genome.
constexpr int kTileN = 64, kTileB = 64, kSampleThreads = 256;

__global__ void __launch_bounds__(kSampleThreads) k_ga_sample(int B, int P, int n,
                                                              const double* __restrict__ ctrl_x,
                                                              const double* __restrict__ genome,
                                                              double* __restrict__ nodes) {
  __shared__ double sN[kTileN][4];
  __shared__ double sx[kTileN];
  __shared__ int ss[kTileN];
  const int i0 = blockIdx.x * kTileN, b0 = blockIdx.y * kTileB;
  const int t = threadIdx.x;
  if (t < kTileN && i0 + t < n) {
    const int i = i0 + t;
    const int nu = (n + 1) / 2;
    const double tp = (i <= nu) ? 0.25 * (1.0 - cos(kPiF64 * i / nu))
                                : 0.5 + 0.25 * (1.0 - cos(kPiF64 * (i - nu) / (n - nu)));
    double N[4];
    const int sp = bspline_basis3(tp, P, N);
    double px = 0.0;
    for (int r = 0; r < 4; ++r) {
      sN[t][r] = N[r];
      px = fma(N[r], ctrl_x[sp - 3 + r], px);
    }
    sx[t] = px;
    ss[t] = sp;
  }
  __syncthreads();
  const int li = t % kTileN;
  const int i = i0 + li;
  if (i >= n) return;
  const int sp = ss[li];
  const double px = sx[li];
  for (int lb = t / kTileN; lb < kTileB; lb += kSampleThreads / kTileN) {
    const int b = b0 + lb;
    if (b >= B) break;
    const double* y = genome + (int64_t)b * P + sp - 3;
    double py = 0.0;
    for (int r = 0; r < 4; ++r) py = fma(sN[li][r], y[r], py);
    const int64_t e = (int64_t)b * n + i;
    nodes[2 * e] = px;
    nodes[2 * e + 1] = py;
  }
}

__global__ void k_ga_step(int B, int P, int k, double p, double pm, const double* __restrict__ lo,
                          const double* __restrict__ hi, const double* __restrict__ sigma,
                          const double* __restrict__ gin, const double* __restrict__ fitness,
                          const double* __restrict__ rand, double* __restrict__ gout) {
  const int pair = blockIdx.x * blockDim.x + threadIdx.x;
  if (pair >= B / 2) return;
  const int R = 4 * k + 5;
  const double* u = rand + (int64_t)pair * R;
  const int pa = tournament(B, k, p, fitness, u);
  const int pb = tournament(B, k, p, fitness, u + 2 * k - 1);
  int c = 1 + (int)floor(__dmul_rn(u[4 * k - 2], (double)(P - 1)));
  if (c > P - 1) c = P - 1;
  const double* A = gin + (int64_t)pa * P;
  const double* Bp = gin + (int64_t)pb * P;
  double* c1 = gout + (int64_t)(2 * pair) * P;
  double* c2 = gout + (int64_t)(2 * pair + 1) * P;
  for (int g = 0; g < P; ++g) {
    c1[g] = (g < c) ? A[g] : Bp[g];
    c2[g] = (g < c) ? Bp[g] : A[g];
  }
  for (int ch = 0; ch < 2; ++ch) {
    const double* um = u + 4 * k - 1 + 3 * ch;
    if (um[0] < pm) {
      int g = (int)floor(__dmul_rn(um[1], (double)P));
      if (g > P - 1) g = P - 1;
      double* x = (ch == 0) ? c1 : c2;
      // rounded as written (no contraction into an FMA): x + sigma (2u - 1)
      const double v = __dadd_rn(x[g], __dmul_rn(sigma[g], __dsub_rn(__dmul_rn(2.0, um[2]), 1.0)));
      x[g] = fmin(fmax(v, lo[g]), hi[g]);
    }
  }
}

// Genome gradient of a loss whose node gradient is grad_nodes: the nodes' y
// coordinates are linear in the genome, y_i = sum_r N_r(t_i) g_r (x fixed), so
// dL/dg_r = sum_i N_r(t_i) dL/dy_i.  One block per airfoil: the basis of every
// node into shared memory, then thread r sums over the nodes in the support of
// control point r in node order (deterministic).  With lr != 0 the genome also
// takes the ascent step g_r <- min(max(g_r + lr dL/dg_r, lo_r), hi_r) where
// dL/dg_r is finite; a gene whose gradient is not (an airfoil whose solve
// failed has NaN node gradients) keeps its value.
constexpr int kGradThreads = 128;

__global__ void __launch_bounds__(kGradThreads) k_ga_genome_grad(
    int P, int n, const double* __restrict__ grad_nodes, double lr, const double* __restrict__ lo,
    const double* __restrict__ hi, double* __restrict__ genome, double* __restrict__ grad_genome) {
  extern __shared__ __align__(16) unsigned char gsm[];
  double* Nb = reinterpret_cast<double*>(gsm);      // n x 4
  double* gy = Nb + 4 * n;                          // n
  int* sp = reinterpret_cast<int*>(gy + n);         // n
  const int b = blockIdx.x;
  const int nu = (n + 1) / 2;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double t = (i <= nu) ? 0.25 * (1.0 - cos(kPiF64 * i / nu))
                               : 0.5 + 0.25 * (1.0 - cos(kPiF64 * (i - nu) / (n - nu)));
    double N[4];
    sp[i] = bspline_basis3(t, P, N);
    for (int r = 0; r < 4; ++r) Nb[4 * i + r] = N[r];
    gy[i] = grad_nodes[2 * ((int64_t)b * n + i) + 1];
  }
  __syncthreads();
  for (int r = threadIdx.x; r < P; r += blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
      const int q = r - (sp[i] - 3);  // index of control point r in node i's four
      if (q >= 0 && q < 4) acc = fma(Nb[4 * i + q], gy[i], acc);
    }
    if (grad_genome) grad_genome[(int64_t)b * P + r] = acc;
    if (lr != 0.0 && isfinite(acc)) {
      double* g = genome + (int64_t)b * P + r;
      *g = fmin(fmax(*g + lr * acc, lo[r]), hi[r]);
    }
  }
}

size_t ga_grad_smem(int n) { return (size_t)n * (4 * 8 + 8 + 4); }

cudaError_t launch_ga_genome_grad(int B, int P, int n, const double* grad_nodes, double lr,
                                  const double* lo, const double* hi, double* genome,
                                  double* grad_genome, cudaStream_t s) {
  const size_t smem = ga_grad_smem(n);
  const cudaError_t e = ensure_smem(k_ga_genome_grad, smem);
  if (e != cudaSuccess) return e;
  k_ga_genome_grad<<<B, kGradThreads, smem, s>>>(P, n, grad_nodes, lr, lo, hi, genome,
                                                 grad_genome);
  return cudaGetLastError();
}

cudaError_t launch_ga_sample(int B, int P, int n, const double* ctrl_x, const double* genome,
                             double* nodes, cudaStream_t s) {
  const dim3 grid((n + kTileN - 1) / kTileN, (B + kTileB - 1) / kTileB);
  k_ga_sample<<<grid, kSampleThreads, 0, s>>>(B, P, n, ctrl_x, genome, nodes);
  return cudaGetLastError();
}

cudaError_t launch_ga_step(int B, int P, int k, double p, double pm, const double* lo,
                           const double* hi, const double* sigma, const double* gin,
                           const double* fitness, const double* rand, double* gout,
                           cudaStream_t s) {
  const int pairs = B / 2;
  k_ga_step<<<(pairs + 127) / 128, 128, 0, s>>>(B, P, k, p, pm, lo, hi, sigma, gin, fitness,
                                                rand, gout);
  return cudaGetLastError();
}

int ga_max_tournament() { return kMaxTournament; }

}  // namespace panel
