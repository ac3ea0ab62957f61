// Householder panel QR of the m_J x b_J leading columns of the trailing
// matrix (the reflector-construction step of Alg. 4 and Alg. 6) and the
// upper-triangular compact-WY factor T with Q = I - Y T Y^T (Sec. 2.2).
//
// One cooperative launch.  CTA g keeps a contiguous range of panel rows in
// shared memory, staged by one TMA 2-D tile load when the panel's layout
// allows it (see launch_panel), else by plain loads.  Column j costs one grid barrier: before it every CTA
// publishes, over its rows below row j, the dot products of column j with
// columns j..b_J-1 (the j-th entry is the squared tail norm), and the owner
// of row j publishes that row.  After it every CTA adds the partial sums in
// the same fixed order (while 56 or more columns remain, in two levels: the
// last CTA of each group of 8 to publish has added its group's partials, in
// CTA order, before the barrier, and every CTA adds the groups' sums), so all
// CTAs derive the same reflector
//   beta = -sign(alpha) ||x||, tau = (beta - alpha)/beta, v = x/(alpha - beta),
// and the same w_c = tau v^T a_c = tau (a_jc + (x^T a_c)_tail/(alpha - beta)),
// update their rows, and compute the partial sums of the next column.
// Finally the CTAs publish partial Gram matrices Y^T Y of their rows and add
// them in a fixed order.  T is the inverse of U = striu(Y^T Y) + diag(1/tau)
// (the same T as the column recurrence T(i,i) = tau_i,
// T(0:i, i) = -tau_i T(0:i,0:i) (Y^T Y)(0:i, i)), so its columns are
// independent back-substitutions:
//   x_j = tau_j,  x_r = -tau_r sum_{t=r+1..j} (Y^T Y)(r, t) x_t  (r < j),
// which also holds with tau_r = 0 (a zero row and column); one warp sweeps
// each column, the columns spread over the grid.
#include "panel.cuh"

namespace rq {
namespace {

using namespace pn;

__global__ void __launch_bounds__(NT, 1) panel_kernel(PanelArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  panel_body(a, blockIdx.x, gridDim.x, smem_raw);
}

// The same with the rows staged by a TMA tile load (see launch_panel).
__global__ void __launch_bounds__(NT, 1)
    panel_kernel_tma(const __grid_constant__ CUtensorMap tm, PanelArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  panel_body(a, blockIdx.x, gridDim.x, smem_raw, &tm);
}

}  // namespace

int panel_grid(int64_t mJ, int bJ, int num_sms) {
  // rows per CTA: 32, or 16 for panels of 128 columns, whose per-column work
  // shrinks faster than the reduction over more CTAs grows (measured: 2048 x
  // 128 7.98 against 8.76 us per column; 64-column panels gain nothing)
  const int64_t rows = bJ >= 128 ? 16 : 32;
  int64_t G = (mJ + rows - 1) / rows;
  if (G > num_sms) G = num_sms;
  if (G < 1) G = 1;
  return (int)G;
}

size_t panel_partial_doubles(int grid, int bJ) {
  return (size_t)2 * grid * bJ + (size_t)grid * bJ * bJ + (size_t)bJ * bJ + (size_t)2 * grid * bJ;
}

static size_t panel_smem(int64_t chunk, int bJ) { return pn::panel_smem_bytes(chunk, bJ); }

// dynamic shared memory limit: 227 KB per CTA less the kernel's static arrays
constexpr size_t kPanelSmemLimit = 200 * 1024;
constexpr int kPanelGroup = 8;
// arrival counters that fit after the barrier word in the handle's state area
constexpr int kPanelMaxGroups = 40;

bool panel_fits(int64_t mJ, int bJ, int num_sms) {
  if (bJ < 1 || bJ > MAXB) return false;
  const int G = panel_grid(mJ, bJ, num_sms);
  const int64_t chunk = (mJ + G - 1) / G;
  return panel_smem(chunk, bJ) <= kPanelSmemLimit;
}

cudaError_t launch_panel(const PanelArgs& a, int num_sms, cudaStream_t st) {
  if (a.bJ > MAXB || a.bJ < 1) return cudaErrorInvalidValue;
  const int G = panel_grid(a.mJ, a.bJ, num_sms);
  const int64_t chunk = (a.mJ + G - 1) / G;
  const size_t smem = panel_smem(chunk, a.bJ);
  if (smem > kPanelSmemLimit) return cudaErrorInvalidValue;
  // TMA staging when the tile's alignment rules hold -- base 16-byte aligned,
  // leading dimension even (16-byte column stride), an even row chunk (its
  // first row x 8 bytes a multiple of 16) of at most 256 rows, the shared-
  // memory tile within the limit -- and the CTAs' chunks are long (>= 64
  // rows): there one asynchronous tile beats 256 threads' element loads
  // (measured: 16384-row panels 3-5 % faster), while short panels lose more
  // to the even pitch's bank conflicts than they gain
  const int64_t chunk_t = tma_chunk(chunk);
  const bool tma = chunk >= 64 && (a.ld % 2 == 0) &&
                   ((reinterpret_cast<uintptr_t>(a.P) & 15) == 0) && chunk_t <= 256 &&
                   panel_smem(chunk_t, a.bJ) <= kPanelSmemLimit;
  CUtensorMap tm;
  const bool use_tma =
      tma && tc::make_map_f64_2d(&tm, a.P, (uint64_t)a.mJ, (uint64_t)a.bJ, (uint64_t)a.ld,
                                 (int)chunk_t, a.bJ) == cudaSuccess;
  static std::atomic<uint64_t> attr_done{0}, attr_done_t{0};
  cudaError_t e = use_tma ? ensure_smem_attr(panel_kernel_tma, (int)kPanelSmemLimit, attr_done_t)
                          : ensure_smem_attr(panel_kernel, (int)kPanelSmemLimit, attr_done);
  if (e != cudaSuccess) return e;
  // the column dots' reduction in two levels (groups of 8 CTAs) on grids of
  // 32 CTAs or more: every CTA then reads ceil(G / 8) sums per column instead
  // of G partial sums (the one-level form reads G^2 per column over the grid)
  PanelArgs args = a;
  const int ngrp_g = (G + kPanelGroup - 1) / kPanelGroup;
  args.group = (G >= 32 && ngrp_g <= kPanelMaxGroups) ? kPanelGroup : 0;
  const int ngrp = args.group ? ngrp_g : 0;
  e = cudaMemsetAsync(a.bar, 0, sizeof(GridBarrier) + sizeof(unsigned) * ngrp, st);
  if (e != cudaSuccess) return e;
  if (use_tma) {
    void* params[] = {&tm, &args};
    return cudaLaunchCooperativeKernel((const void*)panel_kernel_tma, dim3((unsigned)G), dim3(NT),
                                       params, panel_smem(chunk_t, a.bJ), st);
  }
  void* params[] = {&args};
  return cudaLaunchCooperativeKernel((const void*)panel_kernel, dim3((unsigned)G), dim3(NT), params,
                                     smem, st);
}

}  // namespace rq
