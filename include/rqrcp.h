/*
 * rqrcp.h -- C ABI of the GB300 (sm_103a) implementation of randomized QR
 * with column pivoting, its truncated form and the TUXV approximate SVD
 * (Duersch & Gu, "Randomized QR with Column Pivoting").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Matrices are column-major FP64 in device memory; element (i, j) of a
 *   matrix X with leading dimension ldx lives at X[i + j * ldx].
 * - All matrix/vector pointers are DEVICE pointers owned by the caller.  They
 *   must stay valid until the work enqueued on the handle's stream has run.
 * - Every call is asynchronous on the handle's stream (the stream passed to
 *   rqrcp_create or rqrcp_set_stream; NULL means the legacy default stream).
 *   It validates its arguments on the host, enqueues kernels and returns.
 * - Return value: RQRCP_OK when the work was enqueued.  A negative value -i
 *   names the invalid argument i (1-based, the handle is argument 1).
 *   RQRCP_ERR_CUDA reports a CUDA runtime error at enqueue time
 *   (rqrcp_last_error gives the text), RQRCP_ERR_ALLOC a failed workspace
 *   allocation, RQRCP_ERR_UNSUPPORTED a size outside the limits stated below.
 * - Numerical status is a device word, read with rqrcp_sync_info (which
 *   synchronises the stream): 0, or an OR of the RQRCP_INFO_* bits.
 * - Column indices in jpvt are 0-based: jpvt[c] is the original index of the
 *   column that ends up in position c (A[:, jpvt] = Q R).
 * - Omega, the Gaussian compression matrix, is generated on the device from
 *   `seed` by Philox4x32-10 (Salmon et al., SC'11): entry (i, r) of the
 *   l x m matrix uses key (seed mod 2^32, seed >> 32) and counter
 *   (r mod 2^32, r >> 32, i / 2, 1); words (x0,x1) and (x2,x3) give
 *   u = (top 52 bits + 1/2) * 2^-52 and Box-Muller gives rows 2q (cosine)
 *   and 2q+1 (sine).
 * - The handle owns all scratch memory (grown on demand with cudaMalloc;
 *   rqrcp_reserve pre-allocates it).  One handle must not be used from two
 *   host threads at once, and two calls on one handle must not overlap on
 *   the device (they share the scratch); calls on one stream never do.
 *
 * Size limits of this build (RQRCP_ERR_UNSUPPORTED beyond them): b <= 128,
 * l = b + p <= 192; the sample of one block (l x (n - j0)) and the panel of
 * one block ((m - j0) x b) are held in the shared memory of at most one
 * cooperative CTA per SM, which bounds l * n <= 152 * 25000 and
 * m * b <= 152 * 25000 (FP64 elements).
 */
#ifndef RQRCP_H_
#define RQRCP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RQRCP_OK 0
#define RQRCP_ERR_CUDA 1000
#define RQRCP_ERR_ALLOC 1001
#define RQRCP_ERR_UNSUPPORTED 1002
#define RQRCP_ERR_BATCH 1003  /* a problem of trqrcp_batched failed its checks (see last_error) */
#define RQRCP_ERR_BUSY 1004   /* rqrcp_server_submit: the ring slot is still in use */

#define RQRCP_INFO_NONFINITE 1  /* the sample held NaN/Inf: A is not finite */
#define RQRCP_INFO_RESAMPLED 2  /* exactly singular R11: trailing sample re-drawn */
#define RQRCP_INFO_TIMEOUT 4    /* a device-side wait gave up; results invalid */
#define RQRCP_INFO_NOCONV 8     /* the Jacobi SVD of X hit its sweep limit (tuxv_svd) */

typedef struct rqrcp_handle_s* rqrcp_handle_t;

/* Create a handle bound to `cuda_stream` (a cudaStream_t, may be NULL) on the
 * current CUDA device.  Allocates a few kilobytes of device state. */
int rqrcp_create(rqrcp_handle_t* handle, void* cuda_stream);

/* Free the handle and its scratch memory (synchronises its stream first). */
int rqrcp_destroy(rqrcp_handle_t handle);

/* Rebind the handle to another stream. */
int rqrcp_set_stream(rqrcp_handle_t handle, void* cuda_stream);

/* Scratch bytes a call needs: op = 'R' (rqrcp_factor, rqrcp_factor_host),
 * 'Q' (qr_factor), 'T' (trqrcp), 'U' (tuxv, tuxv_iter, tuxv_svd),
 * 'P' (qrcp_factor), 'M' (rqrcp_factor_mixed), 'V' (trqrcp_mixed),
 * 'X' (rqrcp_gemm_f64x: m x n output, k the inner size), 'G'
 * (rqrcp_gemm_bf16x), 'S' (rqrcp_sketch / rqrcp_sample_qrcp: m = l rows,
 * n columns).  k is ignored for 'R', 'Q', 'M' and 'P'.  The size depends on
 * the handle's options (RQRCP_OPT_FP64_EMULATION, RQRCP_OPT_MAX_SMS):
 * rqrcp_reserve on the handle accounts for them. */
size_t rqrcp_workspace_bytes(char op, int64_t m, int64_t n, int64_t k, int b, int p);

/* Allocate the scratch for a later call now (so that the call itself does
 * not allocate, e.g. before stream capture). */
int rqrcp_reserve(rqrcp_handle_t handle, char op, int64_t m, int64_t n, int64_t k, int b, int p);

/* Handle options (value 0/1, default 0, unless stated).
 * RQRCP_OPT_FP64_EMULATION: run the sketch and the two large products of the
 * FP64 trailing update (rqrcp_factor, qr_factor; blocks of b <= 64) on the
 * BF16 tensor cores with the FP64-accurate slicing of rqrcp_gemm_f64x instead
 * of the FP64 pipe.  Its scratch adds 16 bytes per element of A.
 * RQRCP_OPT_RESAMPLE: rqrcp_factor runs Alg. 5 (RSRQRCP) -- before every block
 * after the first, a fresh seeded GIID sample of the updated trailing matrix
 * (Philox stream 0x100 + J after block J) replaces the sample update of
 * Eq. (3); the paper's comparison for the cost of repeated sampling.
 * RQRCP_OPT_MAX_SMS (value = a number of SMs, 0 = all, the default): every
 * launch of the handle's calls uses at most that many CTAs per wave: grids of
 * the cooperative kernels, the persistent tensor-core GEMMs and their split-K
 * choice.  Calls of several handles on separate streams then share the GPU
 * instead of each filling it (the serving slots use this).  Set it before
 * rqrcp_reserve: the scratch size depends on it.  -3 for a negative value. */
#define RQRCP_OPT_FP64_EMULATION 1
#define RQRCP_OPT_RESAMPLE 2
#define RQRCP_OPT_MAX_SMS 3
/* RQRCP_OPT_TEST_BARRIER_TIMEOUT (test of the failure path only, value 0/1):
 * while set, rqrcp_sample_qrcp on this handle launches its cooperative kernel
 * with a grid barrier that waits for one CTA more than the grid has and gives
 * up after a few milliseconds of polling.  The kernel then ORs
 * RQRCP_INFO_TIMEOUT into the status word, writes no-exchange partners
 * (d_swaps[i] = i) for the steps it did not take, leaves dB unchanged and
 * returns; the handle stays usable.  No other call reads the option. */
#define RQRCP_OPT_TEST_BARRIER_TIMEOUT 4
/* RQRCP_OPT_BATCH_TEAM (value 8, 16 or 32; default 16): CTAs per team of the
 * persistent batched kernel (trqrcp_batched, rqrcp_server_*).  A problem's
 * result depends on it (the order of the panel's and the products' partial
 * sums), and on nothing else of the batch.  Larger samples and panels need
 * larger teams: RQRCP_ERR_UNSUPPORTED / RQRCP_ERR_BATCH name the problems that
 * do not fit.  -3 for another value. */
#define RQRCP_OPT_BATCH_TEAM 5
int rqrcp_set_option(rqrcp_handle_t handle, int option, int value);

/* Wait for the handle's stream, then return the device status word in *info
 * and clear it. */
int rqrcp_sync_info(rqrcp_handle_t handle, int* info);

/* Text of the last CUDA error seen by the handle ("" if none). */
const char* rqrcp_last_error(rqrcp_handle_t handle);

/* Text for a return code or info bit. */
const char* rqrcp_status_string(int code);

/*
 * Full randomized QR with column pivoting -- Alg. 4 (RQRCP) of the paper with
 * the sample update of Eq. (3), k = min(m, n).
 *   m, n   : matrix size, m >= 1, n >= 1
 *   dA     : in/out, m x n, lda >= max(1, m).  On exit R is on and above the
 *            diagonal and the Householder vectors (unit leading entry
 *            implied) below it, LAPACK dgeqp3 layout.
 *   b      : block size (pivots per block), 1 <= b <= 128; clamped to k
 *   p      : oversampling, p >= 0; sample rank l = b + p
 *   seed   : Philox seed of Omega
 *   d_jpvt : out, n int64 (0-based permutation, see above)
 *   d_tau  : out, min(m, n) reflector coefficients (H = I - tau v v^T)
 */
int rqrcp_factor(rqrcp_handle_t handle, int64_t m, int64_t n, double* dA, int64_t lda, int b,
                 int p, uint64_t seed, int64_t* d_jpvt, double* d_tau);

/*
 * rqrcp_factor for a matrix in host memory: the same factorization, with the
 * host <-> device copies overlapped with the computation.  The matrix goes up
 * in column chunks on a second stream of the handle, and each chunk's part of
 * the sketch B = Omega A starts when the chunk has landed; after each group of
 * blocks the columns that are final (those left of the current block: later
 * blocks only touch and permute trailing columns) go back while the next
 * blocks run.  The handle's stream completes only after every copy.
 *   hA, ldha : in, host, m x n column-major, ldha >= m
 *   dA, lda  : device work matrix, m x n, lda >= m; holds the factor on exit
 *   b, p, seed : as in rqrcp_factor
 *   hF, ldhf : out, host, m x n (ldhf >= m): R and the reflectors, as in dA;
 *              may be hA itself (every upload precedes every download)
 *   h_jpvt   : out, host, n int64;  h_tau : out, host, min(m, n) doubles
 * Host buffers should be page-locked (cudaHostAlloc / cudaHostRegister) for
 * the copies to overlap; pageable memory works but serialises them.  hA and
 * hF in page-locked memory are moved by a copy kernel reading or writing the
 * mapped host memory (it keeps full speed where the first copy-engine transfer
 * after seconds of computation does not); other memory by the copy engine.  The
 * first call (or a larger n) allocates the device pivots and tau.  Results
 * are available after the handle's stream is synchronised.
 * Errors: -i for argument i (hA is 4, hF 11).
 */
int rqrcp_factor_host(rqrcp_handle_t handle, int64_t m, int64_t n, const double* hA,
                      int64_t ldha, double* dA, int64_t lda, int b, int p, uint64_t seed,
                      double* hF, int64_t ldhf, int64_t* h_jpvt, double* h_tau);

/*
 * Mixed-precision RQRCP (Alg. 4 with Eq. 3) on an FP32 matrix.
 * The sketch B = Omega A is a BF16 product with FP32 accumulation (it only
 * steers pivots); the trailing update W = T^T Y^T A2, A2 -= Y W runs as
 * split-BF16 x3 tensor-core products (rqrcp_gemm_bf16x, FP32-level); the
 * sample QRCP generates its reflectors and downdates its norms in FP64 (the
 * BF16-accurate sample itself is held and transformed in FP32), and the
 * Householder panel, T and the sample update stay in FP64; R's diagonal is
 * returned in FP64.
 *   dA     : in/out, m x n FP32, lda >= m; on exit R (FP32-rounded) on and
 *            above the diagonal and the reflectors below it
 *   d_jpvt : out, n int64;  d_tau : out, min(m, n) FP64
 *   d_rdiag: out, min(m, n) FP64 diagonal of R
 * Exactly singular R11 sets RQRCP_INFO_RESAMPLED and keeps S12 as the next
 * sample rows (this mode does not re-draw the sample).
 */
int rqrcp_factor_mixed(rqrcp_handle_t handle, int64_t m, int64_t n, float* dA, int64_t lda, int b,
                       int p, uint64_t seed, int64_t* d_jpvt, double* d_tau, double* d_rdiag);

/*
 * Unpivoted blocked Householder QR: Alg. 4 with every sample operation and
 * pivot removed (the paper's `qr`, note to Table 3).  dA in/out as in
 * rqrcp_factor (LAPACK dgeqrf layout); d_tau out, min(m, n).
 */
int qr_factor(rqrcp_handle_t handle, int64_t m, int64_t n, double* dA, int64_t lda, int b,
              double* d_tau);

/*
 * Truncated RQRCP without trailing update -- Alg. 6 (TRQRCP).  A is read
 * only; its columns are gathered through the permutation instead of moved
 * (the same result as permuting A in place, Alg. 6, without the copy).
 *   k      : rank, 1 <= k <= min(m, n)
 *   d_jpvt : out, n int64; the first k entries are the selected columns
 *   d_tau  : out, k
 *   dY     : out, m x k, ldy >= m: reflectors, unit diagonal and zeros above
 *            it stored explicitly
 *   dR     : out, k x n, ldr >= k: upper trapezoidal R in the permuted column
 *            order, A[:, jpvt] ~= (I - Y T Y^T)[:, :k] R
 */
int trqrcp(rqrcp_handle_t handle, int64_t m, int64_t n, const double* dA, int64_t lda, int64_t k,
           int b, int p, uint64_t seed, int64_t* d_jpvt, double* d_tau, double* dY, int64_t ldy,
           double* dR, int64_t ldr);

/*
 * Mixed-precision TRQRCP (Alg. 6) on an FP32 matrix: BF16 sketch, the
 * products with A, Y and W^T as split-BF16 x3 tensor-core GEMMs; the sample
 * QRCP's reflectors and norm downdates, the panel, T and R's diagonal in FP64
 * (the sample held and transformed in FP32).  Outputs as in trqrcp with dY (m x k, ldy)
 * and dR (k x n, ldr) in FP32, d_tau and d_rdiag (k) in FP64.
 */
int trqrcp_mixed(rqrcp_handle_t handle, int64_t m, int64_t n, const float* dA, int64_t lda,
                 int64_t k, int b, int p, uint64_t seed, int64_t* d_jpvt, double* d_tau,
                 float* dY, int64_t ldy, float* dR, int64_t ldr, double* d_rdiag);

/*
 * One problem of trqrcp_batched: the arguments of trqrcp_mixed.
 */
typedef struct rqrcp_problem {
  int64_t m, n, k;
  int b, p;
  uint64_t seed;
  const float* dA;
  int64_t lda;
  int64_t* d_jpvt;
  double* d_tau;
  float* dY;
  int64_t ldy;
  float* dR;
  int64_t ldr;
  double* d_rdiag;
} rqrcp_problem;

/*
 * Many uneven-size mixed-precision TRQRCP problems (Alg. 6, the served
 * low-rank workload) in ONE persistent cooperative launch.  The paper factors
 * one matrix at a time; this is the batched form of its truncated algorithm.
 * The grid is divided into teams of G CTAs (RQRCP_OPT_BATCH_TEAM, one CTA per
 * SM); each team claims the next problem from a device copy of `probs`
 * (sorted longest-first by algorithmic flops) and runs all of Alg. 6 on it:
 * Omega from Philox stream 1 with an FP32 Box-Muller transform, the sample
 * B = Omega A and every product with A, Y and W^T as FP32 products on the CUDA
 * cores, the sample QRCP's reflectors and norm downdates (the sample held and
 * transformed in FP32), the Householder panel, T and the sample update of
 * Eq. (3) in FP64.  Outputs per problem are laid out as trqrcp_mixed's (jpvt,
 * tau and rdiag FP64; Y and R FP32); they agree with trqrcp_mixed within FP32
 * rounding, not bit for bit (its products use the split-BF16 tensor-core GEMM).
 * A problem's result depends only on the problem and G: it is the same alone
 * and in any batch.
 *   probs : host array of nprob problem descriptions, copied (through the
 *           handle's page-locked staging buffer) to the device on the
 *           handle's stream; the device buffers they point to must not overlap
 *   teams : problems run at once (0 = as many teams as the handle's SM budget,
 *           RQRCP_OPT_MAX_SMS, holds)
 * Every problem is checked before anything is enqueued: a failing problem
 * returns RQRCP_ERR_BATCH (its index and status in rqrcp_last_error).
 * Limits: b <= 128, b + p <= 192, the sample of one block (l x n) and the panel
 * (m x b) held in the shared memory of the team's G CTAs (about 200 KB each).
 * Device conditions of all problems are ORed into the handle's info word.
 * The call waits for the previous call's table copy before it refills the
 * staging buffer (except during stream capture); team scratch and the device table
 * grow on demand (a device allocation, not allowed during capture): reserve
 * them first with rqrcp_reserve_batched.  A captured launch reads the staging
 * buffer when it runs, so replay it before the next trqrcp_batched call on the
 * same handle.
 */
int trqrcp_batched(rqrcp_handle_t handle, int nprob, const rqrcp_problem* probs, int teams);

/*
 * Sizes the persistent batched kernel's scratch for `teams` teams (0 = as
 * many as fit) and problems up to m x n with rank k, block b, oversampling p,
 * and its descriptor table for 1024 problems.
 */
int rqrcp_reserve_batched(rqrcp_handle_t handle, int teams, int64_t m, int64_t n, int64_t k,
                          int b, int p);

/*
 * Serving loop on the persistent batched kernel (continuous batching; the
 * paper has no serving layer).  rqrcp_server_start launches the kernel of
 * trqrcp_batched on the handle's stream with a request ring in page-locked
 * host memory mapped into the device's address space instead of a fixed
 * table: its teams claim requests as the host publishes them, so requests
 * that arrive while others run are admitted as soon as a team is free, and
 * each request's result is the one trqrcp_batched gives it (the same alone
 * and in any mix).  No graph capture or launch sits on a request's path.
 *   capacity : ring slots (requests published but not yet finished)
 *   teams    : concurrent requests (0 = as many as the handle's SM budget
 *              holds; fewer leave SMs free for other work, e.g. producing the
 *              inputs)
 *   m, n, k, b, p : the largest request the server accepts (scratch sizes)
 * The handle's stream is occupied until the server stops; the teams leave the
 * kernel after about 0.2-0.5 s without requests, and rqrcp_server_submit or
 * rqrcp_server_poll starts it again when needed.  Errors: -i for argument i,
 * RQRCP_ERR_UNSUPPORTED if a server already runs on the handle.
 */
int rqrcp_server_start(rqrcp_handle_t handle, int capacity, int teams, int64_t m, int64_t n,
                       int64_t k, int b, int p);

/*
 * Publishes one request (the fields of rqrcp_problem; device buffers that
 * stay valid and untouched until the request is finished) and returns its
 * ticket.  RQRCP_ERR_BUSY when the ring slot still holds an unfinished
 * request (poll, then retry); RQRCP_ERR_UNSUPPORTED for a request larger than
 * the server's sizes; -2 for an invalid request.
 */
int rqrcp_server_submit(rqrcp_handle_t handle, const rqrcp_problem* prob, int64_t* ticket);

/*
 * 1 when request `ticket` is finished (its outputs are in device memory and
 * *info holds its RQRCP_INFO_* bits), 0 while it is not; -2 for an unknown or
 * reused ticket.  Does not wait.
 */
int rqrcp_server_poll(rqrcp_handle_t handle, int64_t ticket, int* info);

/*
 * Asks the server to stop: its teams leave once the ring is empty.
 * Synchronise the handle's stream to wait for them.
 */
int rqrcp_server_stop(rqrcp_handle_t handle);

/*
 * Deterministic QR with column pivoting, A P = Q R (Alg. 1's pivoting: the
 * column of largest trailing norm at every step), computed with the level-3
 * reflection blocking of Quintana-Orti et al. that the paper describes as the
 * best deterministic scheme (Sec. 2, Alg. qrcp3).  The comparison point for
 * rqrcp_factor: every pivot still needs one pass over the whole trailing
 * matrix (the level-2 inner products y^T A), which the sample avoids.
 *   dA     : in/out, m x n column-major, lda >= m; out: R on and above the
 *            diagonal, reflectors below (LAPACK xGEQP3 layout)
 *   b      : block size (clamped to [1, min(m, n)] and to 128)
 *   d_jpvt : out, n int64 (device), original column index at each position
 *   d_tau  : out, min(m, n) doubles (device)
 * Norm downdates follow LAPACK xLAQP2/xLAQPS: a norm that lost too many digits
 * is recomputed exactly (by ending the block there).  Ties between equal
 * norms go to the lowest position.  Unlike the other calls, this one waits for
 * the device once per block (the block length is read back), so it cannot be
 * captured in a CUDA graph (RQRCP_ERR_UNSUPPORTED during capture).
 * Errors: -i for argument i.
 */
int qrcp_factor(rqrcp_handle_t handle, int64_t m, int64_t n, double* dA, int64_t lda, int b,
                int64_t* d_jpvt, double* d_tau);

/*
 * Approximate truncated SVD -- Alg. 7 (TUXV) with j_max = 1:
 * TRQRCP, Z0 = R P^T, V from the QR of Z0^T, Z1 = A V, [U, X] = qr(Z1).
 *   dU : out, m x k, ldu >= m, orthonormal columns
 *   dX : out, k x k, ldx >= k, upper triangular (zeros below stored)
 *   dV : out, n x k, ldv >= n, orthonormal columns;  A ~= U X V^T
 */
int tuxv(rqrcp_handle_t handle, int64_t m, int64_t n, const double* dA, int64_t lda, int64_t k,
         int b, int p, uint64_t seed, double* dU, int64_t ldu, double* dX, int64_t ldx,
         double* dV, int64_t ldv);

/*
 * Alg. 7 (TUXV) with jmax >= 1 iterations.  After V1 as in tuxv, odd
 * iterations j compute Z = A V and [U, X] = qr(Z) (X upper triangular); even
 * iterations compute Z = U^T A and its LQ factorization [X, V^T] = lq(Z),
 * taken as the QR of Z^T = A^T U (X = R^T lower triangular).  The loop stops
 * after iteration jmax, so X is upper triangular for odd jmax and lower for
 * even jmax; A ~= U X V^T either way.  tuxv is tuxv_iter with jmax = 1.
 * Arguments as in tuxv, with jmax (>= 1) the 10th.  Every iteration is one
 * m x n x k product with A and one k-column QR plus Q formation on the device.
 */
int tuxv_iter(rqrcp_handle_t handle, int64_t m, int64_t n, const double* dA, int64_t lda,
              int64_t k, int b, int p, uint64_t seed, int jmax, double* dU, int64_t ldu,
              double* dX, int64_t ldx, double* dV, int64_t ldv);

/*
 * Approximate truncated SVD: tuxv_iter followed by the SVD of the small
 * connection matrix, X = Ux diag(sigma) Vs^T (Alg. 7 discussion: the diagonal
 * of X approximates the leading singular values, its SVD does better).  The
 * outputs are U Ux, sigma and V Vs, so A ~= U diag(sigma) V^T.
 *   d_sigma : out, k doubles (device), descending, >= 0
 *   dU, dV  : out as in tuxv (orthonormal columns; the column of U belonging
 *             to an exactly zero singular value is 0)
 * The SVD of X is one-sided Jacobi (column-pair rotations, parallel circle
 * ordering, up to 40 sweeps; RQRCP_INFO_NOCONV in the info word if they run
 * out).  Entries of X are assumed below 1e150 in magnitude (their squares are
 * summed unscaled).
 */
int tuxv_svd(rqrcp_handle_t handle, int64_t m, int64_t n, const double* dA, int64_t lda,
             int64_t k, int b, int p, uint64_t seed, int jmax, double* dU, int64_t ldu,
             double* d_sigma, double* dV, int64_t ldv);

/*
 * The Gaussian compression matrix of Alg. 4 (first steps): writes the
 * rows x cols block of the seeded GIID matrix for Philox stream `stream_id`
 * (1 = Omega) into dOut (column-major, ldo >= rows).
 */
int rqrcp_gaussian(rqrcp_handle_t handle, uint64_t seed, uint32_t stream_id, int64_t rows,
                   int64_t cols, double* dOut, int64_t ldo);

/*
 * The initial sample of Alg. 4: B = Omega A with Omega = rqrcp_gaussian(seed,
 * 1, l, m).  dB out, l x n, ldb >= l.
 */
int rqrcp_sketch(rqrcp_handle_t handle, int64_t m, int64_t n, const double* dA, int64_t lda,
                 int ell, uint64_t seed, double* dB, int64_t ldb);

/*
 * Split-BF16 tensor-core GEMM, the contraction engine of the mixed-precision
 * path: C = alpha op(A) op(B) + beta C with FP32 operands and result
 * (column-major; transA/transB 'N' or 'T').  slices = 3 splits each operand
 * element into three bfloat16 parts and sums the six largest slice products
 * with FP32 accumulation in tensor memory (FP32-level accuracy); slices = 1
 * rounds the operands to bfloat16 (one product, FP32 accumulation).
 */
int rqrcp_gemm_bf16x(rqrcp_handle_t handle, char transA, char transB, int64_t m, int64_t n,
                     int64_t k, float alpha, const float* dA, int64_t lda, const float* dB,
                     int64_t ldb, float beta, float* dC, int64_t ldc, int slices);

/*
 * The pivot-selection step of Alg. 4 on its own: partial QRCP (Alg. 1 halted
 * after `steps` pivots) of the ell x nc sample dB (ldb >= ell), in place.
 * On exit dB holds S = Q_b^T B P in the permuted column order (S11 upper
 * triangular with exact zeros below its diagonal, then S12 over S22) and
 * d_swaps[i] (0-based) is the column exchanged with column i at step i.
 * 1 <= steps <= min(ell, nc); ell <= 192.
 */
int rqrcp_sample_qrcp(rqrcp_handle_t handle, int ell, int64_t nc, int steps, double* dB,
                      int64_t ldb, int64_t* d_swaps);

/*
 * Allocation-free form of rqrcp_sample_qrcp (the paper has no counterpart:
 * this is a deployment variant).  For callers that cannot allocate device
 * memory -- code running during CUDA graph stream capture, latency-critical
 * loops that must stay out of the driver's allocator, processes whose device
 * memory is owned by a pool or arena -- it runs the same sample QRCP with its
 * scratch in a fixed device array compiled into the library (about 477 KB,
 * held by every GPU that loads the library until exit), so it needs no
 * handle and calls no cudaMalloc/cudaFree.
 *   ell, nc, steps, dB, ldb, d_swaps : as rqrcp_sample_qrcp (ell <= 192)
 *   d_info      : device int, required; RQRCP_INFO_* bits are ORed into it
 *                 (the caller clears it): RQRCP_INFO_NONFINITE for a sample
 *                 holding NaN or Inf, RQRCP_INFO_TIMEOUT when a grid wait
 *                 gave up (dB and d_swaps are then not a valid result)
 *   cuda_stream : the cudaStream_t to run on (NULL = legacy default stream)
 * Returns -i for an invalid argument i (-7 for a NULL d_info),
 * RQRCP_ERR_UNSUPPORTED when the sample does not fit the kernel's shared
 * memory, RQRCP_ERR_CUDA on a CUDA error.
 * The first call on a device looks up the array's device address; make it
 * before any stream capture.  All calls share the array: calls that overlap on
 * the GPU race, so order them (for example on one stream).
 */
int rqrcp_sample_qrcp_noalloc(int ell, int64_t nc, int steps, double* dB, int64_t ldb,
                              int64_t* d_swaps, int* d_info, void* cuda_stream);

/*
 * FP64-accurate GEMM on the BF16 tensor cores: C = alpha op(A) op(B) + beta C
 * in FP64 (column-major, transA/transB 'N' or 'T').  Each row of op(A) and
 * column of op(B) is scaled by a power of two and cut into seven exact 8-bit
 * BF16 slices; the 28 significant slice products are accumulated on the
 * tensor cores in exact per-diagonal FP32 sums (drained every 64 k into
 * error-free double-FP32 running sums), so the result carries about 48
 * significant bits relative to sum_k |a_ik b_kj|.
 */
int rqrcp_gemm_f64x(rqrcp_handle_t handle, char transA, char transB, int64_t m, int64_t n,
                    int64_t k, double alpha, const double* dA, int64_t lda, const double* dB,
                    int64_t ldb, double beta, double* dC, int64_t ldc);

/*
 * Instrumentation (no counterpart in the paper).  While enabled, every phase
 * of a call is bracketed by CUDA events recorded on the handle's stream, and
 * the algorithmic FLOP count and the number of kernel launches of each phase
 * are accumulated:
 *   0 Omega generation and sketch B = Omega A      4 trailing update (W, A2 -= Y W)
 *   1 sample QRCP                                  5 sample update (Eq. 3)
 *   2 column permutation                           6 TRQRCP/TUXV products
 *   3 panel QR and T factor                        7 other (fills, copies)
 * rqrcp_profile(h, 1) clears the totals and starts recording; (h, 0) stops.
 * rqrcp_profile_read synchronises the stream and writes, for each of the
 * first nphase phases (<= 8), the device milliseconds, algorithmic FLOPs and
 * kernel launches since the last enable; any pointer may be NULL.
 */
/*
 * Arithmetic-peak probe (instrumentation, no counterpart in the paper): one
 * launch of `grid` CTAs x 256 threads on `cuda_stream` that runs `iters`
 * rounds of independent multiply-adds and writes one value per thread to
 * d_sink (device, grid * 256 doubles; floats for kind 3).  *flops receives
 * the launch's floating-point operation count, so that the caller's CUDA
 * event time gives the rate:
 *   kind 0  FP64 FMA on the CUDA cores (8 independent chains per thread)
 *   kind 1  FP64 tensor-core mma.sync m8n8k4 (4 independent tiles per warp)
 *   kind 2  FP64 tensor-core mma.sync m16n8k16 (2 independent tiles per warp)
 *   kind 3  FP32 FMA on the CUDA cores
 *   kind 4  FP64 FMA in a GEMM's register-blocked outer-product pattern
 *           (4 x 4 accumulators per thread, operands renewed every round)
 * Returns -i for an invalid argument i, RQRCP_ERR_CUDA for a launch error.
 */
int rqrcp_peak_probe(int kind, int64_t iters, int grid, void* d_sink, void* cuda_stream,
                     double* flops);

#define RQRCP_NPHASE 8
int rqrcp_profile(rqrcp_handle_t handle, int enable);
int rqrcp_profile_read(rqrcp_handle_t handle, int nphase, double* ms, double* flops,
                       int64_t* launches);

/*
 * Phase times of the persistent batched kernel (instrumentation): while
 * profiling is enabled (rqrcp_profile), the leader CTA of every team adds the
 * wall time of each phase of Alg. 6 to a device counter; this call
 * synchronises the stream and writes, for the first nphase phases (<= 8, the
 * phase numbers of rqrcp_profile; phase 7 includes waiting for a problem),
 * the team-milliseconds summed over all teams since profiling was enabled.
 */
int rqrcp_batched_profile(rqrcp_handle_t handle, int nphase, double* team_ms);

#ifdef __cplusplus
}
#endif

#endif /* RQRCP_H_ */
