// Tiled storage of the inverse velocity blocks of large Vanka patches.
//
// A block of a patch with m velocity DoFs per component is cut into
// nT = ceil(m / 32) tile rows of 32 x 32 tiles; the lower tiles (I, J),
// J <= I, are stored one after another in the order I(I+1)/2 + J, 1024
// elements each.  Diagonal tiles are stored whole (both triangles), entries
// in rows or columns >= m are zero.  Inside a tile, element (r, c) sits at
// r * 32 + (c ^ r): a warp reading one row per lane (row sweep) or one
// column per lane (column sweep) touches 32 different banks either way.
#pragma once
#include <cstdint>

namespace sd {

constexpr int kMaxNp = 4;  // seeds (pressure DoFs) per patch supported by the Vanka kernels
constexpr int kTileElems = 1024;

// Packed block length rounded up to 16 bytes, so every block starts aligned.
template <typename T>
__host__ __device__ __forceinline__ int padded_pk(int m) {
  constexpr int V = 16 / sizeof(T);
  return (m * (m + 1) / 2 + V - 1) / V * V;
}

// Position of key in the ascending list v[0..n), or -1.
__device__ __forceinline__ int bsearch_int(const int* v, int n, int key) {
  int lo = 0, hi = n - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int x = v[mid];
    if (x == key) return mid;
    if (x < key) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

__host__ __device__ __forceinline__ int tile_rows(int m) { return (m + 31) >> 5; }

__host__ __device__ __forceinline__ int64_t tiled_block_elems(int m) {
  const int n = tile_rows(m);
  return (int64_t)n * (n + 1) / 2 * kTileElems;
}

// Offset of element (a, b), a >> 5 >= b >> 5, inside a tiled block.
__host__ __device__ __forceinline__ int tiled_offset(int a, int b) {
  const int I = a >> 5, J = b >> 5, r = a & 31, c = b & 31;
  return ((I * (I + 1) >> 1) + J) * kTileElems + (r << 5) + (c ^ r);
}

}  // namespace sd
