// Launchers of the device kernels (internal interface between the .cu files
// and the host orchestrator in rqrcp.cu).  All launches are asynchronous on
// `st` and return the cudaError_t of the launch.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"

namespace rq {

// ---- philox.cu: seeded GIID matrix (Omega and re-samples)
// Writes rows x cols into out (ld >= rows).  When gate != nullptr the kernel
// does nothing unless *gate != 0.
cudaError_t launch_gaussian(uint64_t seed, uint32_t stream_id, int64_t rows, int64_t cols,
                            double* out, int64_t ld, const int* gate, cudaStream_t st);
// The same rows x cols matrix stored transposed (element (i, r) at out[r + i ld],
// ld >= cols).
cudaError_t launch_gaussian_t(uint64_t seed, uint32_t stream_id, int64_t rows, int64_t cols,
                              double* out, int64_t ld, cudaStream_t st);

// ---- gemm_f64.cu: C = alpha op(A) op(B) + beta C (column-major FP64).
// amode: how A is read -- 0 plain, 1 unit-lower-trapezoidal (entries above the
// diagonal read as 0, diagonal as 1: a Householder block Y stored in place),
// 2 upper-triangular (entries below the diagonal read as 0).
// transA/transB: 'N' or 'T'.  gate: if non-null the kernel runs only when
// *gate == gate_run.  Split-K uses `partial` scratch (splits * M * N doubles)
// when splits > 1.
struct GemmArgs {
  char transA, transB;
  int amode;
  int64_t M, N, K;
  double alpha;
  const double* A;
  int64_t lda;
  const double* B;
  int64_t ldb;
  double beta;
  double* C;
  int64_t ldc;
  const int* gate;
  int gate_run;
  const int64_t* bcols;  // transB == 'N' only: column j of op(B) is stored column bcols[j]
};
cudaError_t launch_gemm(const GemmArgs& g, int splits, double* partial, cudaStream_t st);
int gemm_pick_splits(int64_t M, int64_t N, int64_t K, int num_sms);

// ---- tc_gemm.cu: split-BF16 tensor-core GEMM (tcgen05), FP32 operands.
// The operands are first split into bfloat16 slices (k-contiguous rows of
// op(A) and columns of op(B), in the caller's scratch), then multiplied by a
// persistent TMA-fed kernel.
struct TcGemmArgs {
  char transA, transB;
  int64_t M, N, K;
  float alpha;
  const float* A;
  int64_t lda;
  const float* B;
  int64_t ldb;
  float beta;
  float* C;
  int64_t ldc;
  int* status;
  const int64_t* bcols;  // transB == 'N' only: column j of op(B) is stored column bcols[j]
  __nv_bfloat16* slA;    // >= tc_slice_elems(M, K, slices) elements
  size_t slcapA;
  __nv_bfloat16* slB;    // >= tc_slice_elems(N, K, slices) elements
  size_t slcapB;
  float* partial;        // split-K sums (2 floats per element of C and split); may be null
  size_t partial_cap;    // floats
  int num_sms;
};
// slices = 1 (plain BF16) or 3 (FP32-level split, six products)
cudaError_t launch_tc_gemm(TcGemmArgs g, int slices, cudaStream_t st);
size_t tc_slice_elems(int64_t rows, int64_t K, int slices);
// kernel launches one launch_tc_gemm call makes
int tc_launches(int64_t M, int64_t N, int64_t K, int num_sms, size_t partial_cap);

// ---- oz_gemm.cu: FP64-accurate GEMM on the BF16 tensor cores by exact
// slicing.  C (M x N, FP64, ldc) = alpha * 2^(expA_i + expB_j) * (A_sl B_sl^T)
// + beta * C, where A_sl and B_sl are the slices written by launch_oz_slice
// (rows of op(A) and columns of op(B), oz_slice_elems(rows, K) bf16 each).
struct OzGemmArgs {
  int64_t M, N, Kp;
  const __nv_bfloat16* As;
  const int* expA;
  const __nv_bfloat16* Bs;
  const int* expB;
  double alpha, beta;
  double* C;
  int64_t ldc;
  int* status;
  float* partial;      // split-K sums (2 floats per element of C and split); may be null
  size_t partial_cap;  // floats
  int num_sms;
};
// Slices of the R rows of op(X) (K values each): kc -> row r is stored column
// r (X[k + r ld]), else stored row r (X[r + k ld]); amode 1 reads X as a
// unit-lower reflector block.  slices: oz_slice_elems(R, K) bf16; exps: R ints,
// the biased FP64 exponent field of each row's largest |x| (the row scale).
cudaError_t launch_oz_slice(const double* X, int64_t ld, bool kc, int amode, int64_t R, int64_t K,
                            __nv_bfloat16* slices, int* exps, cudaStream_t st);
cudaError_t launch_oz_gemm(const OzGemmArgs& g, cudaStream_t st);
int64_t oz_kpad(int64_t K);
size_t oz_slice_elems(int64_t rows, int64_t K);
// kernel launches of one launch_oz_slice call
int oz_slice_launches(bool kc, int64_t K);
// kernel launches of one launch_oz_gemm call
int oz_launches(int64_t M, int64_t N, int64_t Kp, int num_sms, size_t partial_cap);

// ---- sample_qrcp.cu: partial QRCP (Alg. 1, b steps) on the l x nc sample.
struct SampleQrcpArgs {
  double* B;          // l x nc, leading dimension ldb; overwritten by S in the permuted order
  int64_t ldb;        // >= ell
  int ell;
  int64_t nc;
  int steps;          // bJ
  int64_t* swaps;     // out: steps entries, partner position of each swap
  double* cand;       // scratch: 2 * grid * 4 doubles (key, position, alpha, sigma2)
  double* candcol;    // scratch: 2 * grid * l doubles
  GridBarrier* bar;
  int* status;
  // test of the device-side timeout only: the grid barrier waits for this
  // many extra CTAs that do not exist (with a poll bound of a few ms), so the
  // first barrier runs out, RQRCP_INFO_TIMEOUT is set and every CTA returns
  int phantom = 0;
  // nonzero: the sample is held and the reflectors applied in FP32 (a sample
  // that is single-precision accurate to begin with); the reflectors are
  // generated and the norms downdated in FP64 either way
  int f32 = 0;
};
cudaError_t launch_sample_qrcp(const SampleQrcpArgs& a, int num_sms, cudaStream_t st);
bool sample_qrcp_fits(int ell, int64_t nc, int num_sms);

// ---- permute.cu: apply the swap sequence of one block to whole columns.
// A: m rows, columns col0 + (0..nc); swaps relative to col0.  jpvt (may be
// null) moves alongside.  `map` scratch: 1 + 10 * steps int64, `buf` scratch:
// m * 2 * steps doubles.  m may be 0 (then only jpvt moves).
cudaError_t launch_apply_swaps(double* A, int64_t lda, int64_t m, int64_t col0,
                               const int64_t* swaps, int steps, int64_t* jpvt, int64_t* map,
                               double* buf, cudaStream_t st);
cudaError_t launch_apply_swaps_f32(float* A, int64_t lda, int64_t m, int64_t col0,
                                   const int64_t* swaps, int steps, int64_t* jpvt, int64_t* map,
                                   float* buf, cudaStream_t st);
cudaError_t launch_iota(int64_t* v, int64_t n, cudaStream_t st);
cudaError_t launch_convert_f32_f64(const float* src, int64_t lds, double* dst, int64_t ldd,
                                   int64_t rows, int64_t cols, cudaStream_t st);
cudaError_t launch_convert_f64_f32(const double* src, int64_t lds, float* dst, int64_t ldd,
                                   int64_t rows, int64_t cols, cudaStream_t st);
cudaError_t launch_gather_cols_f32(const float* src, int64_t lds, int64_t r0, int64_t rows,
                                   const int64_t* idx, int64_t ncols, float* dst, int64_t ldd,
                                   cudaStream_t st);
// dst (cols x cols, ldd) = upper triangle of src (zeros below)
cudaError_t launch_copy_upper_f32(const float* src, int64_t lds, int64_t cols, float* dst,
                                  int64_t ldd, cudaStream_t st);
cudaError_t launch_panel_writeback(const double* P, int64_t ldp, int64_t rows, int64_t cols,
                                   float* A, int64_t lda, float* Y, int64_t ldy, double* rdiag,
                                   cudaStream_t st);
// dst(:, t) = src(r0:r0+rows, idx[t]) for t < ncols (column gather through a map)
cudaError_t launch_gather_cols(const double* src, int64_t lds, int64_t r0, int64_t rows,
                               const int64_t* idx, int64_t ncols, double* dst, int64_t ldd,
                               cudaStream_t st);
// dst(idx[c], r) = src(r, c): scatter-transpose of a rows x ncols block
cudaError_t launch_scatter_transpose(const double* src, int64_t lds, int64_t rows,
                                     const int64_t* idx, int64_t ncols, double* dst, int64_t ldd,
                                     cudaStream_t st);
// Y(:, c) explicit from in-place storage F (rows x cols): unit diagonal,
// zeros above, F below; R part (upper triangle, zeros below) into Rout.
cudaError_t launch_split_qr(const double* F, int64_t ldf, int64_t rows, int64_t cols, int64_t yrow0,
                            double* Y, int64_t ldy, double* Rout, int64_t ldr, cudaStream_t st);
// dst(r, c) = src(r, c), rows x cols, one side page-locked host memory that is
// mapped into the device address space (a copy made by the SMs)
cudaError_t launch_copy_mapped(const double* src, int64_t lds, double* dst, int64_t ldd,
                               int64_t rows, int64_t cols, cudaStream_t st);
// X = R^T (lower triangular, zeros above) for the upper triangle R of F's
// leading cols x cols block
cudaError_t launch_r_transposed(const double* F, int64_t ldf, int64_t cols, double* X,
                                int64_t ldx, cudaStream_t st);

// ---- panel.cu: Householder panel QR (unblocked, cooperative) of the
// mJ x bJ panel P (ld), tau out, T (bJ x bJ, ld bJ) the compact-WY factor.
struct PanelArgs {
  double* P;
  int64_t ld;
  int64_t mJ;
  int bJ;
  double* tau;
  double* T;          // out, bJ x bJ, column-major, zeros below the diagonal
  double* partial;    // scratch: panel_partial_doubles(grid, bJ) doubles
  double* rowj;       // scratch: 2 bJ doubles
  // with group > 1, ceil(grid / group) unsigned arrival counters follow the
  // barrier word (zeroed with it by the launcher)
  GridBarrier* bar;
  int* status;
  // mixed precision: round the reflectors below the diagonal to FP32 values
  // before the Gram, and set tau_i = 2 / v_i^T v_i (kept 0 where the column
  // had a zero tail), so that T and tau describe exactly the stored vectors
  int round_f32;
  // the column dots' grid reduction in two levels: the last CTA of each group
  // of `group` consecutive CTAs to publish adds the group's partial sums, and
  // every CTA then adds the groups' sums (0 or 1: every CTA adds all CTAs'
  // partial sums).  launch_panel sets it (8 for grids of 32 CTAs or more);
  // the barrier word must then be followed by ceil(grid / 8) unsigned ints.
  int group = 0;
};
cudaError_t launch_panel(const PanelArgs& a, int num_sms, cudaStream_t st);
size_t panel_partial_doubles(int grid, int bJ);
int panel_grid(int64_t mJ, int bJ, int num_sms);
bool panel_fits(int64_t mJ, int bJ, int num_sms);

// ---- sample_update.cu: W11 = S11 R11^{-1} (bJ x bJ, ld bJ).  Sets *flag to 1
// (and ORs RQRCP_INFO_RESAMPLED into status) when R11 has an exact zero
// diagonal entry, else 0.
cudaError_t launch_w11(const double* S, int ell, const double* R11, int64_t ldr, int bJ,
                       double* W11, int* flag, int* status, cudaStream_t st);

// ---- svd_jacobi.cu: X = Ux diag(sigma) Vs^T for a k x k matrix X (one-sided
// Jacobi, cooperative when the grid has more than one CTA).  Ux, Vs, G, Vx
// are k x k with ld k; sigma descending.  A column of Ux whose singular value
// is exactly 0 is left 0.  RQRCP_INFO_NOCONV is ORed into *status when the
// sweeps run out before every pair is orthogonal.
constexpr int kJacobiMaxSweeps = 40;
struct JacobiArgs {
  const double* X;
  int64_t ldx;
  int k;
  double* G;       // scratch, the rotated copy of X
  double* Vx;      // scratch, the accumulated rotations
  double* Ux;      // out
  double* Vs;      // out
  double* sigma;   // out, k
  double* sraw;    // scratch, k
  int* rotated;    // scratch, kJacobiMaxSweeps ints
  GridBarrier* bar;
  int* status;
};
cudaError_t launch_jacobi_svd(const JacobiArgs& a, int num_sms, cudaStream_t st);
int jacobi_grid(int k, int num_sms);

// ---- qrcp3.cu: deterministic QRCP with level-3 reflection blocking (the
// paper's comparison method).  One cooperative launch factors up to bJ
// columns starting at position i0 of the m x n matrix A (column-major, lda),
// whose columns [i0, n) are up to date on rows >= i0.  Writes R rows, the
// reflectors (LAPACK layout below the diagonal), tau, W(c, t) (n x kQrcp3MaxB
// region used as n x bJ, ld n) and ctl[1] = the number of columns done (fewer
// than bJ when a norm downdate lost too many digits).  The caller then applies
// A(i0+nb:, i0+nb:) -= Y W^T.
constexpr int kQrcp3MaxB = 128;
constexpr int kQrcp3Chunks = 16;
constexpr int64_t kQrcp3SmemRows = 24576;  // rows of the reflector staged in shared memory
struct Qrcp3Args {
  double* A;
  int64_t lda;
  int64_t m, n;
  int64_t i0;
  int bJ;
  double* vn1;        // n, trailing column norms (downdated)
  double* vn2;        // n, norms at their last exact computation
  int* redo;          // n, nonzero: recompute the norm at the next block start
  int64_t* jpvt;      // n, original column index at each position
  double* tau;        // >= min(m, n)
  double* W;          // n x bJ, ld n
  double* ys;         // m, the current column before scaling
  double* dots;       // kQrcp3Chunks x n partial inner products
  long long* cand;    // 2 per CTA
  double* npart;      // 1 per CTA
  int* ctl;           // [0] stop flag, [1] columns done
  GridBarrier* bar;
  int* status;
  int64_t smem_rows;  // set by the launcher
};
cudaError_t launch_qrcp3_block(const Qrcp3Args& a, int num_sms, cudaStream_t st);
size_t qrcp3_smem_bytes(int64_t m);

// ---- batched.cu: persistent batched mixed-precision TRQRCP (Alg. 6) --
// teams of G co-resident CTAs claim problems from a device table or from a
// request ring in mapped host memory and run the whole algorithm on each.
// Byte offsets of the per-team scratch areas.
struct BatchLayout {
  size_t ctl, omega, B, Wt, P64, T, T32, Z32, YY, W11, swaps, map, cbuf, jbuf, cand, candcol,
      ppart, rowj, part;
  int64_t part_elems;  // floats in `part`
};
// Largest problem a team's scratch must hold.
struct BatchLimits {
  int64_t m, n, k;
  int b, ell;
};
// Request ring of the serving loop, in page-locked host memory mapped into
// the device's address space.  Followed in memory by `cap` rqrcp_problem
// slots, `cap` (rounded up to even) int info words and `cap` int64 done words
// (ticket + 1 once the request is finished).  The host publishes a request
// by writing its slot, then raising `tail` (release order).
struct RequestRing {
  long long tail;  // requests published
  int stop;        // nonzero: teams exit once the ring is empty
  int cap;         // slots
  int running;     // set by the host at launch; 0 once every team has exited
  int pad0;
  long long pad[5];
};
size_t request_ring_bytes(int cap);
struct BatchLaunch {
  const rqrcp_problem* table;  // device table (batch mode) or nullptr
  int nprob;
  RequestRing* ring;           // device address of the mapped ring (serving) or nullptr
  unsigned long long* next;    // claim counter
  int* exited;                 // teams that have left the loop (serving)
  int G, teams;
  char* scratch;
  size_t team_bytes;
  BatchLayout L;
  GridBarrier* bars;           // teams entries
  int* status;
  unsigned int idle_polls;     // serving: polls of an empty ring before a team exits
  int keep_next;               // serving relaunch: tickets continue from the counter
  long long* trace;            // 8 phase times (ns) per team, accumulated; null = off
};
size_t batch_team_bytes(const BatchLimits& lim, int G, BatchLayout* L);
bool batch_fits(int64_t m, int64_t n, int b, int ell, int G);
cudaError_t launch_batch_trqrcp(const BatchLaunch& bl, cudaStream_t st);

// Q = first cols columns of the rows x rows identity
cudaError_t launch_eye(double* Q, int64_t rows, int64_t cols, int64_t ld, cudaStream_t st);
// Fill / copy helpers
cudaError_t launch_fill(double* X, int64_t rows, int64_t cols, int64_t ld, double v,
                        cudaStream_t st);
cudaError_t launch_copy2d(const double* src, int64_t lds, double* dst, int64_t ldd,
                          int64_t rows, int64_t cols, cudaStream_t st);

}  // namespace rq
