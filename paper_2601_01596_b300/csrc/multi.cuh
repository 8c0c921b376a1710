// multi.cuh -- one launch of a loop pass over every shape group of a plan.
//
// A batch of uneven items (Alg. 1 per item; 2D/3D items of several shapes,
// 1D items of several Bluestein splits) is grouped by shape, and each group's
// pass is normally one launch over its members.  The multi-group form runs a
// pass kind for ALL groups in one persistent launch: the plan holds a device
// work list of units (group, member, tile block), every unit being one CTA's
// work of that group's plain kernel; a grid of as many CTAs as fit on the
// device walks the list (unit u, u + gridDim.x, ...) and each CTA runs the
// body of the unit's group, selected by the group's transform length.  The
// bodies are the plain passes' own (k_px_body, k_axis_body, k_chk_body,
// k1_col_body, k1_row_body), so every item sees exactly the arithmetic of
// its separate launch, and a member that has stopped returns at once (its
// item's predicate, as in the separate launches).
//
// Every unit runs 128 threads: the tile widths of the multi-group form are
// those whose CTA is 128 threads at every length (strided passes 8 pencils,
// 4 at length 1024; contiguous passes one warp per tile).
#pragma once
#include "bluestein.cuh"
#include "passes.cuh"

namespace ffcz {

constexpr int kMultiGroups = 8;   // groups one multi-group launch covers
constexpr int kMultiThreads = 128;
enum MultiKind : int { MK_PX = 0, MK_YINV = 1, MK_YFWD = 2, MK_CHK = 3, MK_COL1 = 4, MK_ROW1 = 5, MK_N = 6 };

// Tile widths of the multi-group form.
__host__ __device__ constexpr int multi_w_strided(int L) { return L >= 1024 ? 4 : 8; }
__host__ __device__ constexpr int multi_w_rows(int L) { return 32 / (1 << (ilog2(L) / 2)) > 0 ? 32 / (1 << (ilog2(L) / 2)) : 1; }

struct MultiArgs {
  Args a[kMultiGroups];        // the pass's arguments for each group
  int32_t len[kMultiGroups];   // the pass's transform length for each group
  const int2* units;           // work list: {group | member << 4, tile block}
  int64_t nunits;
};

// One unit of a group of length L.  Not inlined: each length's body gets its
// own register allocation (inlined into one switch, the bodies of all
// lengths shared one allocation and spilled far more).
template <int KIND, int L>
__device__ __noinline__ void multi_unit(const Args& a, int bx, int by) {
  if constexpr (KIND == MK_PX) k_px_body<float, L, multi_w_rows(L), false, PV_POCS, false>(a, bx, by);
  else if constexpr (KIND == MK_YINV) k_axis_body<float, L, +1, multi_w_strided(L)>(a, bx, by);
  else if constexpr (KIND == MK_YFWD) k_axis_body<float, L, -1, multi_w_strided(L)>(a, bx, by);
  else if constexpr (KIND == MK_CHK) k_chk_body<float, L, multi_w_strided(L), false, PV_POCS, false>(a, bx, by);
  else if constexpr (KIND == MK_COL1) k1_col_body<float, L, multi_w_strided(L)>(a, bx, by);
  else k1_row_body<float, L, multi_w_rows(L)>(a, bx, by);
}

template <int KIND>
__global__ void __launch_bounds__(kMultiThreads, 3) k_multi(const __grid_constant__ MultiArgs m) {
  for (int64_t u = blockIdx.x; u < m.nunits; u += gridDim.x) {
    const int2 wu = m.units[u];
    const int g = wu.x & 15, gi = wu.x >> 4, bx = wu.y;
    __syncthreads();   // the previous unit's shared-memory reads are done
    switch (m.len[g]) {
      case 8: multi_unit<KIND, 8>(m.a[g], bx, gi); break;
      case 16: multi_unit<KIND, 16>(m.a[g], bx, gi); break;
      case 32: multi_unit<KIND, 32>(m.a[g], bx, gi); break;
      case 64: multi_unit<KIND, 64>(m.a[g], bx, gi); break;
      case 128: multi_unit<KIND, 128>(m.a[g], bx, gi); break;
      case 256: multi_unit<KIND, 256>(m.a[g], bx, gi); break;
      case 512: multi_unit<KIND, 512>(m.a[g], bx, gi); break;
      case 1024: multi_unit<KIND, 1024>(m.a[g], bx, gi); break;
      default: break;
    }
  }
}

// Host side: the grid of one group's pass in the multi-group form (the same
// CTA decomposition as its separate launch at the multi-group tile width),
// and the dynamic shared memory of one unit.
struct MultiGrid {
  int64_t gx;    // CTAs per member
  size_t smem;   // bytes
};

template <int KIND, int L>
MultiGrid multi_grid_of(int64_t extent_a, int64_t extent_b) {
  // extent_a, extent_b: px (rows, -); axis (Nz, M); chk (M, Nmid);
  // col1 (P2, -); row1 (P1, -)
  constexpr bool rows_kind = KIND == MK_PX || KIND == MK_ROW1;
  constexpr int W = rows_kind ? multi_w_rows(L) : multi_w_strided(L);
  using G_ = Geo<float, L, W>;
  static_assert(G_::NTHR == kMultiThreads, "multi-group units run 128 threads");
  int64_t tiles = 0;
  if constexpr (KIND == MK_PX || KIND == MK_ROW1) tiles = (extent_a + W - 1) / W;
  else if constexpr (KIND == MK_YINV || KIND == MK_YFWD) tiles = extent_a * (extent_b / W);
  else if constexpr (KIND == MK_CHK) tiles = chk_ntiles(W, (int)extent_a, (int)extent_b);
  else tiles = extent_a / W;
  MultiGrid r;
  r.gx = (tiles + G_::G - 1) / G_::G;
  r.smem = KIND == MK_PX ? Smem<float, L, W>::bytes_x : Smem<float, L, W>::bytes_axis;
  return r;
}

}  // namespace ffcz
