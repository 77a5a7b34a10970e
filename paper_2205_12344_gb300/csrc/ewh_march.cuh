// Device helpers shared by the marching step kernels (ewh_zmarch.cu: 3D,
// along z; ewh_ymarch.cu: 2D, along y): mbarrier and bulk-tensor PTX, the
// scaled SBP first derivative (12 D) with its exact reach per row, and the
// per-class tap tables that let every lane of a warp run the same code on
// closure rows.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ewh_internal.cuh"

namespace ewh {
namespace {

constexpr int ZM_CLASSES = 9;  // SBP rows of a line position: 0..3 low side, 4 interior, 5..8 high side

static_assert(SBP_CLOSURE[0][4] == 0.0 && SBP_CLOSURE[0][5] == 0.0 && SBP_CLOSURE[1][1] == 0.0 &&
                  SBP_CLOSURE[1][3] == 0.0 && SBP_CLOSURE[1][4] == 0.0 && SBP_CLOSURE[1][5] == 0.0 &&
                  SBP_CLOSURE[2][2] == 0.0 && SBP_CLOSURE[2][5] == 0.0 && SBP_CLOSURE[3][1] == 0.0 &&
                  SBP_CLOSURE[3][3] == 0.0,
              "the closure taps below skip exactly the zero entries of the SBP boundary block");

// ---- PTX helpers: shared-memory addresses, mbarriers, bulk tensor copies --
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long zm_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Request one u plane (3 components of box ZM_UX x UY at padded (cx, cy, cz),
// components cc .. cc + 2) into dst; completion is counted on bar.
__device__ __forceinline__ void zm_issue(const CUtensorMap* tm, float* dst, uint64_t* bar, int cx, int cy, int cz,
                                         int cc, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(cx), "r"(cy), "r"(cz), "r"(cc), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void zm_pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void zm_pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---- the SBP first derivative, scaled by 12 --------------------------------
__device__ __forceinline__ float c4u(float m2, float m1, float p1, float p2) { return (m2 - p2) + 8.0f * (p1 - m1); }

// First and last line positions read by the difference at p (line of n >= 8
// nodes): the exact reach of each row of D (closure rows 0..3 read columns
// {0,1,2,3}, {0,2}, {0,1,3,4}, {0,2,4,5}; the interior p +- 2).
__device__ __forceinline__ int zm_lo(int p, int n) {
  if (p < 4) return 0;
  if (p > n - 5) {
    const int r = n - 1 - p;
    return n - 1 - (r == 0 ? 3 : r == 1 ? 2 : r == 2 ? 4 : 5);
  }
  return p - 2;
}
__device__ __forceinline__ int zm_hi(int p, int n) {
  if (p < 4) return p == 0 ? 3 : p == 1 ? 2 : p == 2 ? 4 : 5;
  if (p > n - 5) return n - 1;
  return p + 2;
}

// The last line position p in [lo, cap] whose stencil is complete once
// position `done` exists, for a segment whose first stencil reaches h0: the
// largest such p with max(h0, zm_hi(p, n)) <= done (the reach's prefix
// maximum, non-decreasing in p), or a value below lo when there is none.  In
// the interior (done in [6, n - 3]) that is done - 2, without the search.
__device__ __forceinline__ int zm_last_ready(int lo, int cap, int h0, int done, int n) {
  if (h0 <= done && done >= 6 && done <= n - 3) return min(cap, done - 2);
  int p = min(cap, done);
  while (p >= lo && max(h0, zm_hi(p, n)) > done) --p;
  return p;
}

__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ void st2(float* p, float a, float b) { *reinterpret_cast<float2*>(p) = make_float2(a, b); }

// The closure rows of 12 D (p < 4 or p > n - 5); v(o) is the value at offset o.
template <class F>
__device__ __forceinline__ float zm_closure12(F v, int p, int n, const float* tab) {
  const bool low = p < 4;
  const int r = low ? p : n - 1 - p;
  auto w = [&](int j) { return low ? v(j - p) : v(n - 1 - j - p); };
  float d;
  switch (r) {
    case 0: d = tab[0] * w(0) + tab[1] * w(1) + tab[2] * w(2) + tab[3] * w(3); break;
    case 1: d = tab[6] * w(0) + tab[8] * w(2); break;
    case 2: d = tab[12] * w(0) + tab[13] * w(1) + tab[15] * w(3) + tab[16] * w(4); break;
    default: d = tab[18] * w(0) + tab[20] * w(2) + tab[22] * w(4) + tab[23] * w(5); break;
  }
  return low ? d : -d;
}


// Class of line position p (0 <= p < n): 0..3 low SBP rows, 4 interior (also
// used outside the line, where the result is discarded), 5..8 high rows.
__device__ __forceinline__ int zm_class(int p, int n) {
  if (p < 0 || p >= n) return 4;
  if (p < 4) return p;
  if (p > n - 5) return 5 + (n - 1 - p);
  return 4;
}

// 12 D at a node of class c from the four taps of the table (v at the node,
// `stride` between line neighbours): the same code for every lane.
__device__ __forceinline__ float zm_d12t(const float* v, int stride, int c, const int* toff, const float* tcf) {
  const int4 o = *reinterpret_cast<const int4*>(toff + 4 * c);
  const float4 w = *reinterpret_cast<const float4*>(tcf + 4 * c);
  return w.x * v[o.x * stride] + w.y * v[o.y * stride] + w.z * v[o.z * stride] + w.w * v[o.w * stride];
}


// ---- host side --------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}


// The four taps of 12 D per class (offsets from the node, weights): the
// nonzero columns of each closure row (mirrored and negated from the high
// side), the interior row, zero-weight padding.
inline void zm_class_taps(int* toff, float* tcf) {
  static const int kCols[4][4] = {{0, 1, 2, 3}, {0, 2, -1, -1}, {0, 1, 3, 4}, {0, 2, 4, 5}};
  for (int c = 0; c < ZM_CLASSES; ++c)
    for (int q = 0; q < 4; ++q) {
      int off = 0;
      double w = 0.0;
      if (c == 4) {
        static const int io[4] = {-2, -1, 1, 2};
        static const double iw[4] = {1.0, -8.0, 8.0, -1.0};
        off = io[q];
        w = iw[q];
      } else {
        const int r = c < 4 ? c : c - 5;
        const int j = kCols[r][q];
        if (j >= 0) {
          off = c < 4 ? j - r : r - j;
          w = (c < 4 ? 12.0 : -12.0) * SBP_CLOSURE[r][j];
        }
      }
      toff[4 * c + q] = off;
      tcf[4 * c + q] = (float)w;
    }
}

// Tile origin shift along one axis.  A tile's stress halo reaches 2 nodes and
// its u tile 4 nodes beyond it, which covers every difference except where a
// tile ends within 5 nodes of the high side: a stress node on SBP row n - 4
// at the halo's last position reads u 3 further, and an own node on row n - 4
// or n - 1 reads stresses 3 away.  That happens exactly when the last tile
// holds 2 or 4 unknowns (Dirichlet high side) or 1, 3 or 5 (traction-free).
// Starting the tiles `sh` nodes before the first unknown changes the last
// tile's count; sh is the least multiple of `step` that avoids those counts.
inline int zm_shift(int nu, int tile, bool hi_free, int step) {
  for (int sh = 0; sh < tile; sh += step) {
    const int last = (nu + sh) % tile == 0 ? tile : (nu + sh) % tile;
    const bool bad = hi_free ? (last == 1 || last == 3 || last == 5) : (last == 2 || last == 4);
    if (!bad) return sh;
  }
  return -1;
}

}  // namespace
}  // namespace ewh
