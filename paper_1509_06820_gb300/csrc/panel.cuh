// Householder panel QR with its compact-WY factor T as a device function
// over a group of co-resident CTAs: the body of the cooperative panel kernel,
// shared with the persistent batched kernel.  The algorithm and its data
// layout are described in panel.cu.
#pragma once

#include "kernels.cuh"
#include "tcgen05.cuh"

namespace rq {
namespace pn {

constexpr int NT = 256;
constexpr int MAXB = 128;
constexpr int PARTS = 8;   // threads per column in the partial-sum reduction
constexpr int RB = 40;     // loads in flight per thread in that reduction
constexpr int MAXGROUP = 16;  // largest CTA group of the two-level reduction
// the two-level form pays for its extra round trips (the group's arrival
// counter, its partial sums) only while many columns remain; below it,
// warps 1.. take at most G x 54 / 224 <= 37 sources per thread (one round of
// RB loads)
constexpr int GROUP_MIN_COLS = 56;

// Row chunk of a TMA-staged panel: the plain chunk rounded up to 2 (mod 4).
// Even, so a CTA's first row is 16-byte aligned for the tile load; 2 (mod 4),
// so the tile's pitch spreads a warp's column-strided accesses over eight of
// the sixteen 8-byte banks (an odd pitch, used for plain loads, spreads them
// over all sixteen).
__host__ __device__ inline int64_t tma_chunk(int64_t chunk) { return chunk + ((6 - chunk % 4) % 4); }

// The panel QR and T on CTA g of a group of G co-resident CTAs (the whole
// grid of the standalone kernel, or one team of the persistent batched
// kernel); smem_raw: panel_smem_bytes(chunk, bJ) bytes of dynamic shared memory.
// tmap: when given, the CTA's rows are staged into shared memory by one TMA
// 2-D tile load (box: chunk rows x bJ columns with chunk = tma_chunk(...), the
// tile's pitch chunk); otherwise by plain loads into a layout of odd pitch.
__device__ __forceinline__ void panel_body(const PanelArgs& a, int g, int G,
                                           unsigned char* smem_raw,
                                           const CUtensorMap* tmap = nullptr) {
  const int bJ = a.bJ;
  const int64_t chunk0 = (a.mJ + G - 1) / G;
  const int64_t chunk = tmap ? tma_chunk(chunk0) : chunk0;
  const int64_t r_lo = (int64_t)g * chunk;
  const int nrow = (int)imax64(0, imin64(a.mJ, r_lo + chunk) - r_lo);
  // plain loads: odd pitch, so rows of one column sit in distinct banks; TMA:
  // the box's pitch
  const int64_t ldp = tmap ? chunk : (chunk | 1);
  double* Ps = reinterpret_cast<double*>(smem_raw);  // chunk x bJ, ld = ldp
  __shared__ double s_w[MAXB];
  __shared__ double s_part[PARTS][MAXB];
  __shared__ double s_scal[4];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = NT / 32;

  if (tmap != nullptr) {
    // one TMA tile per CTA (rows past the panel read as zero), completion
    // counted on an mbarrier; the wait is bounded
    __shared__ __align__(8) uint64_t s_mbar;
    if (tid == 0) {
      tc::mbar_init(&s_mbar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
      tc::mbar_expect_tx(&s_mbar, (uint32_t)(chunk * bJ * 8));
      tc::tma_load_2d(Ps, tmap, (int)r_lo, 0, &s_mbar);
    }
    if (!tc::mbar_wait(&s_mbar, 0u)) {
      if (tid == 0) {
        atomicExch(&a.bar->abort, 1u);
        atomicOr(a.status, RQRCP_INFO_TIMEOUT);
      }
      return;
    }
  } else {
    for (int64_t e = tid; e < (int64_t)nrow * bJ; e += NT) {
      const int64_t r = e % nrow, c = e / nrow;
      Ps[r + c * ldp] = __ldcg(a.P + (r_lo + r) + c * a.ld);
    }
  }
  __syncthreads();

  // 2 x G x bJ (column dots), G x bJ x bJ (Gram partials), bJ x bJ (Gram),
  // 2 x ceil(G / group) x bJ (the groups' sums of the column dots)
  double* part_base = a.partial;
  // two-level reduction of the column dots: CTA g belongs to group g / C of
  // cq consecutive CTAs; the last of them to publish adds the group's partial
  // sums in increasing CTA order (no waiting: an arrival counter per group,
  // after the barrier word, says which CTA is last)
  const int C = (a.group > 1 && a.group <= MAXGROUP) ? a.group : 1;
  const int ngrp = (G + C - 1) / C;
  const int grp_q = g / C, grp_q0 = grp_q * C, grp_cq = min(C, G - grp_q0);
  double* gsum_base = part_base + (size_t)2 * G * bJ + (size_t)G * bJ * bJ + (size_t)bJ * bJ;
  unsigned* grp_cnt = reinterpret_cast<unsigned*>(a.bar + 1);
  __shared__ int s_last;
  // partial dots of column j with columns j..bJ-1 over owned rows below row j
  auto publish = [&](int j) {
    double* part = part_base + (size_t)(j & 1) * G * bJ + (size_t)g * bJ;
    const int rstart = (int)imax64(0, (int64_t)j + 1 - r_lo);  // local first row > j
    const int ncols = bJ - j;
    // P lanes per column (a power of two within a warp), as many columns at
    // once as fit in the block; the P partial sums meet by shuffles
    int P = 32;
    while (P > 1 && NT / P < ncols) P >>= 1;
    const int cpr = NT / P;
    const int p = tid % P;
    for (int c0 = 0; c0 < ncols; c0 += cpr) {
      const int c = j + c0 + tid / P;
      double s = 0.0;
      if (c < bJ) {
        const double* xj = Ps + (size_t)j * ldp;
        const double* xc = Ps + (size_t)c * ldp;
        for (int r = rstart + p; r < nrow; r += P) s = fma(xj[r], xc[r], s);
      }
      for (int o = P >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (p == 0 && c < bJ) part[c] = s;
    }
    if (j >= r_lo && j < r_lo + nrow) {
      double* rowj = a.rowj + (size_t)(j & 1) * bJ;
      for (int c = j + tid; c < bJ; c += NT) rowj[c] = Ps[(j - r_lo) + c * ldp];
    }
    if (C > 1 && bJ - j >= GROUP_MIN_COLS) {
      // every group member adds one to the counter per grouped step, so the
      // last of a step sees a multiple of cq, less one
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        const unsigned old = atomicAdd(grp_cnt + grp_q, 1u);
        s_last = (old % (unsigned)grp_cq) == (unsigned)(grp_cq - 1);
      }
      __syncthreads();
      if (s_last) {
        __threadfence();
        const double* pq = part_base + (size_t)(j & 1) * G * bJ + (size_t)grp_q0 * bJ;
        double* gs = gsum_base + ((size_t)(j & 1) * ngrp + grp_q) * bJ;
        for (int c = j + tid; c < bJ; c += NT) {
          double v[MAXGROUP];
#pragma unroll
          for (int u = 0; u < MAXGROUP; ++u) v[u] = u < grp_cq ? __ldcg(pq + (size_t)u * bJ + c) : 0.0;
          double t = v[0];
#pragma unroll
          for (int u = 1; u < MAXGROUP; ++u)
            if (u < grp_cq) t += v[u];
          gs[c] = t;
        }
      }
    }
  };

  publish(0);
  for (int j = 0; j < bJ; ++j) {
    if (!grid_barrier(a.bar, G, a.status)) return;
    // fixed-order reduction of the partial dots (or of the groups' sums).
    // Warp 0 adds column j's sources (lane-strided, then a shuffle tree) and
    // forms the reflector's scalars from them -- a dependent FP64 chain --
    // while warps 1.. add the other columns' sources: PARTS threads per
    // column, thread pp adds sources q = pp, pp + PARTS, ... in increasing
    // order with up to RB loads in flight; the PARTS sums are added in order.
    const int ncols = bJ - j;
    const bool grouped = C > 1 && ncols >= GROUP_MIN_COLS;
    const double* part = grouped ? gsum_base + (size_t)(j & 1) * ngrp * bJ
                                 : part_base + (size_t)(j & 1) * G * bJ;
    const int nsrc = grouped ? ngrp : G;
    const double* rowj = a.rowj + (size_t)(j & 1) * bJ;
    const int nc1 = ncols - 1;                            // columns after j
    const int parts = imin64(PARTS, imax64(1, (NT - 32) / imax64(1, nc1)));
    if (warp == 0) {
      const double alpha = __ldcg(rowj + j);
      double sj = 0.0;
      for (int q = lane; q < nsrc; q += 32) sj += __ldcg(part + (size_t)q * bJ + j);
      sj = warp_sum(sj);
      if (lane == 0) {
        double beta, tau, scale;
        house_scalars_sq(alpha, sj, &beta, &tau, &scale);
        s_scal[0] = beta;
        s_scal[1] = tau;
        s_scal[2] = scale;
        if (g == 0) a.tau[j] = tau;
      }
    } else if (nc1 > 0) {
      for (int c = j + 1 + tid - 32; c < bJ; c += NT - 32) s_w[c] = __ldcg(rowj + c);  // row j
      // warp-uniform rounds; the adds stop at the warp's largest source count
      const int total = parts * nc1;
      for (int e0 = (warp - 1) * 32; e0 < total; e0 += NT - 32) {
        const int e = e0 + lane;
        const bool act = e < total;
        const int c = j + 1 + (act ? e % nc1 : 0), pp = act ? e / nc1 : 0;
        const int cnt = act ? (nsrc - pp + parts - 1) / parts : 0;  // sources pp, pp + parts, ...
        const int cmax = __reduce_max_sync(0xffffffffu, (unsigned)cnt);
        double s = 0.0;
        for (int u0 = 0; u0 < cmax; u0 += RB) {
          double v[RB];
#pragma unroll
          for (int u = 0; u < RB; ++u)
            v[u] = (u0 + u < cnt) ? __ldcg(part + (size_t)(pp + (u0 + u) * parts) * bJ + c) : 0.0;
#pragma unroll
          for (int u = 0; u < RB; ++u) {
            if (u0 + u >= cmax) break;
            if (u0 + u < cnt) s += v[u];
          }
        }
        if (act) s_part[pp][c] = s;
      }
    }
    __syncthreads();
    const double beta = s_scal[0], tau = s_scal[1], scale = s_scal[2];
    // w_c = tau * v^T a_c for c > j (v_j = 1, v_r = scale x_r below)
    for (int c = j + 1 + tid; c < bJ; c += NT) {
      double st = 0.0;
      for (int pp = 0; pp < parts; ++pp) st += s_part[pp][c];
      s_w[c] = tau * (s_w[c] + scale * st);
    }
    const int64_t jl = (int64_t)j - r_lo;  // local index of row j (may be outside)
    const int64_t rstart = imax64(0, jl + 1);
    // scale column j into v, then a_rc -= v_r w_c on owned rows below j
    for (int64_t r = rstart + tid; r < nrow; r += NT) Ps[r + j * ldp] *= scale;
    __syncthreads();
    if (tau != 0.0) {
      // (row, column) pairs packed densely over the threads (32-bit indices)
      const int ncols = bJ - j - 1;
      const int rows = nrow - (int)rstart;
      const double* vj = Ps + (size_t)j * ldp;
      for (int e = tid; e < rows * ncols; e += NT) {
        const int cc = e / rows;
        const int r = (int)rstart + (e - cc * rows);
        const int c = j + 1 + cc;
        Ps[r + (size_t)c * ldp] = fma(-vj[r], s_w[c], Ps[r + (size_t)c * ldp]);
      }
    }
    if (jl >= 0 && jl < nrow) {
      // row j: R entries
      for (int c = j + 1 + tid; c < bJ; c += NT) Ps[jl + c * ldp] -= (tau != 0.0) ? s_w[c] : 0.0;
      if (tid == 0) Ps[jl + j * ldp] = beta;
    }
    __syncthreads();
    if (j + 1 < bJ) publish(j + 1);
  }

  // mixed precision: the stored reflectors are the FP32-rounded ones
  if (a.round_f32) {
    for (int64_t e = tid; e < (int64_t)nrow * bJ; e += NT) {
      const int64_t r = e % nrow, c = e / nrow;
      if (r_lo + r > c) Ps[r + c * ldp] = (double)(float)Ps[r + c * ldp];
    }
    __syncthreads();
  }
  // write the factored rows back
  for (int64_t e = tid; e < (int64_t)nrow * bJ; e += NT) {
    const int64_t r = e % nrow, c = e / nrow;
    a.P[(r_lo + r) + c * a.ld] = Ps[r + c * ldp];
  }
  // partial Gram Y^T Y over owned rows (upper triangle, Y unit lower)
  double* gram = part_base + (size_t)2 * G * bJ + (size_t)g * bJ * bJ;
  for (int e = tid; e < bJ * bJ; e += NT) {
    const int c1 = e % bJ, c2 = e / bJ;  // entry (c1, c2), c1 <= c2
    if (c1 > c2) continue;
    // rows R >= c2 only (y2 is zero above its unit diagonal); the diagonal
    // row of each column reads as 1
    const int64_t r0 = imax64(0, (int64_t)c2 - r_lo);
    double s = 0.0;
    if (r0 < nrow && r_lo + r0 == c2) {
      s = (c1 == c2) ? 1.0 : Ps[r0 + c1 * ldp];
      for (int64_t r = r0 + 1; r < nrow; ++r) s = fma(Ps[r + c1 * ldp], Ps[r + c2 * ldp], s);
    } else {
      for (int64_t r = r0; r < nrow; ++r) s = fma(Ps[r + c1 * ldp], Ps[r + c2 * ldp], s);
    }
    gram[c1 + c2 * bJ] = s;
  }
  if (!grid_barrier(a.bar, G, a.status)) return;
  // every CTA adds the partials of the Gram entries e = g, g + G, ... over all
  // CTAs q in increasing order (PP threads per entry, then a fixed-order
  // combine), so the reduction is spread over the grid
  {
    const double* gp = part_base + (size_t)2 * G * bJ;
    double* gtot = part_base + (size_t)2 * G * bJ + (size_t)G * bJ * bJ;
    const int nent = (bJ * bJ - g + G - 1) / G;   // entries owned by this CTA
    const int PP = nent >= NT ? 1 : (nent * 8 <= NT ? 8 : (nent * 4 <= NT ? 4 : (nent * 2 <= NT ? 2 : 1)));
    __shared__ double s_g[NT];
    for (int i0 = 0; i0 < nent; i0 += NT / PP) {
      const int i = i0 + tid / PP, sub = tid % PP;
      double s = 0.0;
      if (i < nent) {
        const int e = g + i * G;
        for (int q0 = sub; q0 < G; q0 += 8 * PP) {
          double v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int q = q0 + u * PP;
            v[u] = (q < G) ? __ldcg(gp + (size_t)q * bJ * bJ + e) : 0.0;
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) s += v[u];
        }
      }
      s_g[tid] = s;
      __syncthreads();
      if (sub == 0 && i < nent) {
        double t = 0.0;
        for (int u = 0; u < PP; ++u) t += s_g[tid + u];
        gtot[g + i * G] = t;
      }
      __syncthreads();
    }
  }
  if (!grid_barrier(a.bar, G, a.status)) return;
  // ---- T by column back-substitution: column j on CTA j % G, warp j / G
  const int warps_needed = (bJ + G - 1) / G;  // columns per CTA, rounded up
  if (g >= bJ) return;
  const double* gtot = part_base + (size_t)2 * G * bJ + (size_t)G * bJ * bJ;
  // this CTA's largest column decides how much of the Gram it needs
  int jmax = -1;
  for (int j = g; j < bJ; j += G) jmax = j;
  double* Gs = Ps;            // (jmax + 1) x (jmax + 1) upper part, ld bJ
  double* taus = Ps + (size_t)bJ * bJ;  // bJ adjusted tau values
  for (int e = tid; e < (jmax + 1) * bJ; e += NT) {
    const int r = e % bJ, c = e / bJ;
    if (r <= c) Gs[e] = __ldcg(gtot + e);
  }
  // every tau (CTA 0 writes the adjusted ones back in the mixed mode)
  for (int r = tid; r < bJ; r += NT) {
    double t = __ldcg(a.tau + r);
    // mixed precision: tau_r = 2 / v_r^T v_r for the stored (rounded) v_r;
    // zero stays zero
    if (a.round_f32 && t != 0.0) t = 2.0 / __ldcg(gtot + r + (size_t)r * bJ);
    taus[r] = t;
  }
  __syncthreads();
  for (int wq = warp; wq < warps_needed; wq += nwarps) {
    const int j = g + wq * G;
    if (j < bJ) {
      constexpr int RPL = MAXB / 32;  // rows per lane
      double acc[RPL];
#pragma unroll
      for (int q = 0; q < RPL; ++q) acc[q] = 0.0;
      double xt = taus[j];
      double* Tj = a.T + (size_t)j * bJ;
      for (int r = j + 1 + lane; r < bJ; r += 32) Tj[r] = 0.0;
      if (lane == 0) Tj[j] = xt;
      for (int t = j; t >= 1; --t) {
        // acc(r) += G(r, t) x_t for r < t, then x_{t-1} = -tau_{t-1} acc(t-1)
        const double* gt = Gs + (size_t)t * bJ;
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
          const int r = lane + 32 * q;
          if (r < t) acc[q] = fma(gt[r], xt, acc[q]);
        }
        const int rn = t - 1, owner = rn & 31, qn = rn >> 5;
        double mine = 0.0;
#pragma unroll
        for (int q = 0; q < RPL; ++q)
          if (q == qn) mine = acc[q];
        const double val = -taus[rn] * mine;
        xt = __shfl_sync(0xffffffffu, val, owner);
        if (lane == owner) Tj[rn] = xt;
      }
    }
  }
  if (a.round_f32 && g == 0) {
    __syncthreads();
    for (int r = tid; r < bJ; r += NT) a.tau[r] = taus[r];
  }
}

__host__ __device__ inline size_t panel_smem_bytes(int64_t chunk, int bJ) {
  size_t a = (size_t)(chunk | 1) * bJ * 8;
  size_t b = ((size_t)bJ * bJ + bJ) * 8;
  return a > b ? a : b;
}

}  // namespace pn
}  // namespace rq
