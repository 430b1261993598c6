// tl_layout.cuh -- the tiled layout of a large airfoil's factor while the
// step-synchronous LU (k_lu_large.cu, k_update_tc.cu) runs on it.
//
// The caller's factor buffer holds m x m floats per airfoil (m = n + 1) with
// row stride m, which is arbitrary: a row does not start on a 16-byte
// boundary, so the tensor-memory-access (TMA) unit cannot copy tiles of it.
// During the factorisation the airfoil's m^2 floats are therefore kept in a
// different order, in the same place:
//
//   blocks   The rows and columns are cut into T = ceil(m / 128) blocks: a
//            first, ragged block of e = m - 128 (T - 1) in [1, 128] rows, then
//            T - 1 blocks of 128.  Step K of the LU factors block K, so every
//            step after the first one works on whole 128 x 128 tiles.
//   row 0    Block row 0 (the first e rows) stays row-major, row stride m.
//   row I    Block row I >= 1 occupies the same 128 m floats as its rows do in
//            the row-major order.  In it: the first h_I floats of the ragged
//            tile (I, 0) (128 x e, row-major, row stride e), then the full
//            tiles (I, 1) .. (I, T-1), 16384 floats each, then the rest of
//            tile (I, 0).  h_I in [0, 31] is chosen so that the full tiles start
//            on a 128-byte boundary of the buffer.
//   tiles    A full tile is four chunks of 32 columns, each chunk 128 rows of
//            32 floats (128 bytes per row, 16 KB per chunk): element (r, c) at
//            (c / 32) 4096 + 32 r + c % 32.  Once the U12 block of row I is
//            formed (step I), its tiles (I, J > I) hold the transpose: element
//            (r, c) at (r / 32) 4096 + 32 c + r % 32, i.e. chunks of 32 rows of
//            U stored column by column -- the K-major operand the tensor cores
//            read for B.
//
// Viewed as rows of 32 floats, every chunk of every full tile starts on a row
// boundary of one two-dimensional array (the whole factor buffer, 128-byte
// rows), so one tensor map describes every chunk of every airfoil.  After the
// last step the transposed U tiles are turned back to row chunks
// (k_tl_untranspose), and the refinement reads the factor in this layout: a
// row of block row I >= 1 is its ragged part, then 32-float chunks 4096 floats
// apart.
#pragma once
#include <cuda.h>

#include "lu_mixed.cuh"

namespace panel {

constexpr int kTlB = 128;               // block size
constexpr int kTlC = 32;                // chunk width in floats (one 128-byte row)
constexpr int kTlTile = kTlB * kTlB;    // floats per full tile
constexpr int kTlChunk = kTlB * kTlC;   // floats per chunk

struct TlGeom {
  int m;         // matrix size n + 1
  int T;         // number of blocks
  int e;         // size of the first (ragged) block, 1..128
  int64_t base;  // float offset of the airfoil's matrix in the buffer

  __device__ __forceinline__ void init(int m_, int64_t base_) {
    m = m_;
    T = (m + kTlB - 1) / kTlB;
    e = m - kTlB * (T - 1);
    base = base_;
  }
  // first row / column of block I and its size
  __device__ __forceinline__ int start(int I) const { return I == 0 ? 0 : e + kTlB * (I - 1); }
  __device__ __forceinline__ int size(int I) const { return I == 0 ? e : kTlB; }
  // float offset (from base) of block row I's span
  __device__ __forceinline__ int64_t span(int I) const { return (int64_t)start(I) * m; }
  __device__ __forceinline__ int head(int I) const { return (int)((-(base + span(I))) & 31); }
  // float offset (from base) of the full tile (I, J), I, J >= 1
  __device__ __forceinline__ int64_t tile(int I, int J) const {
    return span(I) + head(I) + (int64_t)(J - 1) * kTlTile;
  }
  // float offset (from base) of element (rr, c) of the ragged tile (I >= 1, 0)
  __device__ __forceinline__ int64_t rag(int I, int rr, int c) const {
    const int idx = rr * e + c, hh = head(I);
    return span(I) + (idx < hh ? idx : hh + (int64_t)(T - 1) * kTlTile + (idx - hh));
  }
  // float offset (from base) of element (r, c); `ut`: the tiles (I, J > I) of
  // block row I hold their transpose (true once step I has formed U12)
  __device__ __forceinline__ int64_t off(int r, int c, bool ut) const {
    if (r < e) return (int64_t)r * m + c;
    const int I = 1 + (r - e) / kTlB, rr = (r - e) & (kTlB - 1);
    if (c < e) return rag(I, rr, c);
    const int J = 1 + (c - e) / kTlB, cc = (c - e) & (kTlB - 1);
    const int64_t t = tile(I, J);
    if (ut && J > I) return t + (int64_t)(rr >> 5) * kTlChunk + cc * kTlC + (rr & 31);
    return t + (int64_t)(cc >> 5) * kTlChunk + rr * kTlC + (cc & 31);
  }
};

// The factor buffer as one tensor map (k_update_tc.cu).
struct UpdateMap {
  CUtensorMap map;    // boxes of 128 rows, 128-byte swizzle (a chunk)
  CUtensorMap map32;  // boxes of 32 rows, no swizzle (a quarter of a chunk)
};
cudaError_t make_update_map(float* base, uint64_t floats, UpdateMap* out);
cudaError_t ensure_update_smem();
cudaError_t launch_update_tc(const SolveArgs& a, const UpdateMap& map, int K, int split,
                             long long spin, cudaStream_t s);
cudaError_t launch_trsm_tc(const SolveArgs& a, const UpdateMap& map, int K, int split,
                           long long spin, cudaStream_t s);

}  // namespace panel
