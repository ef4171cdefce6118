/*
 * ctm.h -- C ABI of libctm, a GB300 (sm_103a) implementation of the
 * corner-transfer-matrix (CTM) move for a square-lattice iPEPS with a 2-site
 * {A, B} unit cell, in the standard form and in the reduced-environment,
 * sequential-order form of Lan & Evenbly, "Reduced Contraction Costs of
 * Corner-Transfer Methods for PEPS".
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Site tensors A, B are real, row-major [d][D][D][D][D] with legs (p, u, l, d, r)
 * (Sec. II: physical dimension d, virtual dimension D).  Site (i, j) of the
 * lattice holds A when i + j is even.
 *
 * The environment (Sec. II, Fig. 1d) is stored as 16 tensors (kind, k, x):
 * kind 0 = corner C, 1 = edge T; k = 1 (left / top-left), 2 (top / top-right),
 * 3 (right / bottom-right), 4 (bottom / bottom-left); x = 0 for sublattice a,
 * 1 for b (the site the tensor is adjacent to).  Legs run clockwise around the
 * boundary: corners are [prev][next] (C1[down][right], C2[left][down],
 * C3[up][left], C4[right][up]); edges are [prev][ket][bra][next]
 * (T1[down][k][b][up], T2[left][k][b][right], T3[up][k][b][down],
 * T4[right][k][b][left]).
 *
 * Moves: dir 0 = left, 1 = up, 2 = right, 3 = down.  A move absorbs two
 * columns (Sec. II, Fig. 2a); the up, right and down moves are the left move
 * of the lattice turned counter-clockwise by 1, 2, 3 quarter turns.
 *
 * Errors: every int-returning call returns CTM_OK (0) or a negative code and
 * never aborts the process; ctm_last_error() describes the last failure of a
 * context.  All device work is issued on the stream given to ctm_init_env.
 * Calls on one context must not overlap (the context is not thread-safe).
 */
#ifndef CTM_H
#define CTM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ctm_ctx ctm_ctx;

enum {
  CTM_OK = 0,
  CTM_ERR_ARG = -1,         /* bad argument (size, enum, null pointer) */
  CTM_ERR_OOM = -2,         /* device or host allocation failed */
  CTM_ERR_CUDA = -3,        /* a CUDA runtime call failed */
  CTM_ERR_NAN = -4,         /* a NaN/Inf or zero-norm tensor was produced */
  CTM_ERR_NOCONV = -5,      /* iteration / Jacobi sweep cap reached */
  CTM_ERR_UNSUPPORTED = -6  /* combination not built in this library */
};

enum { CTM_LEFT = 0, CTM_UP = 1, CTM_RIGHT = 2, CTM_DOWN = 3 };
/* CTM_REDUCED_ENV: the intermediate method of Sec. III (reduced environment,
 * 4-index isometry, double-layer absorption, O(chi^3 D^4)). */
enum { CTM_STANDARD = 0, CTM_REDUCED_SEQUENTIAL = 1, CTM_REDUCED_ENV = 2 };
/* Arithmetic of the absorption / renormalisation contractions.  Projector
 * factorisations, normalisation, spectra and observables are FP64 always. */
enum { CTM_FP64 = 0, CTM_TF32 = 1, CTM_BF16 = 2 };
/* OR-ed into `precision` of ctm_init_env: fold only (bond dimension D^2), no
 * growth; for callers that install their own environment with ctm_set_tensor. */
enum { CTM_INIT_NO_GROW = 0x100 };

/*
 * Create a context, copy A and B (host or device pointers, detected with
 * cudaPointerGetAttributes; the caller keeps ownership), and build the
 * initial environment: every tensor is a site whose outward legs are closed by
 * `boundary` (D x D row-major, ket x bra; NULL = identity, i.e. each outward
 * ket leg traced with its bra partner), giving bond dimension D^2; standard
 * moves (Sec. II) then grow every bond to chi (the reduced networks of
 * Sec. III-IV cannot raise a bond above the current one).
 * chi_prime is the intermediate dimension chi' of the split isometries
 * (Sec. IV; the paper uses chi' = chi); pass 0 for chi.
 * stream: a cudaStream_t (NULL = the legacy default stream).
 * The context owns all device memory it allocates; free it with ctm_free.
 */
int ctm_init_env(ctm_ctx** out, const double* A, const double* B, int d, int D,
                 int chi, int chi_prime, int precision, const double* boundary,
                 void* stream);

/*
 * One CTM move in direction dir (Sec. II; mode CTM_STANDARD uses the 8-tensor
 * half-network projector of Fig. 2c, mode CTM_REDUCED_SEQUENTIAL the reduced
 * network of Fig. 3c / Fig. 8 with split isometries and the ket-then-bra
 * absorption of Fig. 4).  Every new tensor is scaled to unit Frobenius norm.
 * Returns CTM_ERR_NAN if a tensor became non-finite or zero.
 */
int ctm_move(ctm_ctx* ctx, int dir, int mode);

/*
 * Repeat iterations of (left, up, right, down) moves until the 8 corner
 * spectra (each scaled to sum s^2 = 1) change by less than tol in 2-norm
 * (maximum over corners), or max_iter iterations ran (Sec. II: N_CTM ~ 10-30).
 * Writes the iterations done and the last change; returns CTM_ERR_NOCONV when
 * max_iter was reached without convergence.
 */
int ctm_converge(ctm_ctx* ctx, int mode, int max_iter, double tol,
                 int* iters_done, double* last_delta);

/*
 * <op> on one nearest-neighbour bond from the 2-site reduced density matrix of
 * the environment (the 2 x 4 window of Sec. II, Fig. 1d; e.g. the Heisenberg
 * bond of Eq. 1 that Sec. V evaluates): bond 0 = a left of b, 1 = b left of a,
 * 2 = a above b, 3 = b above a.  op is host, row-major (d*d) x (d*d) with rows
 * and columns ordered (first site, second site).  The result is written to
 * *value (host).  The ket and bra layers of each site enter one after the other
 * (the order of Sec. IV), so the largest intermediate is chi^2 d^2 D^4 doubles.
 */
int ctm_expect_bond(ctm_ctx* ctx, int bond, const double* op, double* value);

/*
 * Singular values of corner `corner` (0..7 = C1a, C1b, C2a, C2b, C3a, C3b,
 * C4a, C4b), descending and scaled to sum s^2 = 1 (the corner spectra whose
 * change decides convergence, Sec. II).  s is a host buffer of at least chi
 * entries; *len receives the count written.
 */
int ctm_corner_spectrum(ctm_ctx* ctx, int corner, double* s, int* len);

/*
 * All 8 corner spectra at once (same order and scaling as ctm_corner_spectrum;
 * Sec. II), with one batched FP64 Jacobi launch when the corners share a shape.
 * For corners of 64 or more columns that launch runs on C V, V the rotations of
 * a batched FP32 Jacobi run on C made orthonormal in FP64 (the values are those
 * of C; the FP64 run then needs a few sweeps).  s is a host buffer of
 * 8 * maxlen doubles (row i = corner i); lens[8] receives the counts.
 */
int ctm_corner_spectra(ctm_ctx* ctx, double* s, int maxlen, int* lens);

/*
 * Connected correlation along a row (Sec. V, Fig. 9b: S_zz(x)):
 * out[x-1] = <op1_0 op2_x> - <op1_0><op2_x> for x = 1..xmax, sites 0..x of a
 * row starting on sublattice a, from the strip closed by C1_a, T1_a, C4_a on
 * the left and by C2, T3, C3 of site x on the right.  op1, op2: host, d x d
 * row-major; out: host, xmax doubles.  FP64.
 */
int ctm_correlator(ctm_ctx* ctx, const double* op1, const double* op2, int xmax, double* out);

/*
 * Per-site log norm ln kappa = (1/4) ln[Z22 Z00 / (Z20 Z02)] from the 2x2
 * window (Sec. II, Fig. 1d) with top-left site a, where Zhw closes the environment around an
 * h x w block of sites (corner and edge normalisations cancel).  For the
 * Ising-norm PEPS this is ln Z / N.
 */
int ctm_log_kappa(ctm_ctx* ctx, double* value);

/*
 * Copy environment tensor (kind, k, x) -- one of the corner and edge tensors
 * of Sec. II, Fig. 1d -- to the host buffer `out` (may be NULL to query) and its
 * 2 (corner) or 4 (edge) dims to dims[0..3].
 */
int ctm_get_tensor(ctm_ctx* ctx, int kind, int k, int x, double* out, int* dims);

/*
 * Overwrite environment tensor (kind, k, x) (Sec. II, Fig. 1d) from a host
 * buffer with the given dims (2 for a corner, 4 for an edge; bond dims at most
 * chi, ket/bra dims D).
 */
int ctm_set_tensor(ctm_ctx* ctx, int kind, int k, int x, const double* in,
                   const int* dims);

/*
 * Replace the site tensors A and B of a context (same d and D; host or device
 * pointers, copied; Sec. II) and keep its environment: the next moves and
 * observables use the new A, B.  Recorded CUDA graphs are discarded and
 * double-layer tensors already built are rebuilt.
 */
int ctm_set_sites(ctm_ctx* ctx, const double* A, const double* B);

/*
 * Reverse mode (Sec. III-IV and the Appendix, differentiated): the loss
 *   E = (1/4) sum over the 4 bonds of <op>  (the bond observable of
 *       ctm_expect_bond, e.g. the Heisenberg S.S of Eq. 1)
 * evaluated after `iters` iterations (left, up, right, down) of the
 * reduced-sequential move started from the context's current environment,
 * which is held fixed (a constant of the loss) and is not modified; and its
 * gradient with respect to A and B, through every sequential absorption
 * (Fig. 4b), projector application and truncated SVD (Fig. 4a, Fig. 8).
 * Everything runs in FP64 on the device, whatever the context's precision: the
 * truncated SVDs are exact one-sided Jacobi SVDs whose thin factors feed the
 * adjoint of ctm_svd_left_adjoint with Lorentzian broadening eps (relative to
 * s_max^4, e.g. 1e-12).  Each iteration is checkpointed: only the environment
 * entering it is kept, and the backward pass recomputes it.
 * op: host, (d*d) x (d*d) row-major.  energy: host.  gA, gB: d*D^4 doubles each
 * (host or device, may be NULL), laid out like A and B.
 * Errors: CTM_ERR_ARG (iters < 0, eps < 0, null op or energy), CTM_ERR_NAN,
 * CTM_ERR_NOCONV, CTM_ERR_OOM, CTM_ERR_CUDA.
 */
int ctm_energy_grad(ctm_ctx* ctx, int iters, double eps, const double* op, double* energy,
                    double* gA, double* gB);

/* Number of kernels this library launched on the context so far.
 * (Measurement; no counterpart in the paper.) */
long long ctm_kernel_launches(ctm_ctx* ctx);

/*
 * Per-class kernel timing (measurement; no counterpart in the paper) with CUDA
 * events recorded on the context's stream around every launch of a class
 * (0 = FP64 contraction, 1 = TF32 tensor-core contraction, 2 = BF16 tensor-core
 * contraction, 3 = Jacobi SVD sweep kernel, 4 = fused FP64 CholeskyQR, whose
 * flop count, 2 rows n^2 + n^3 / 3 per pass it ran, is summed on the device:
 * a problem stops after its first unshifted pass on a well-conditioned input).
 * ctm_profile_enable(ctx, mask) clears the counters and records the classes
 * whose bit (1 << class) is set in mask; 0 stops.  Changing the mask discards
 * the context's recorded CUDA graphs (they are recaptured with event nodes for
 * the timed classes at the next steady-state moves).
 * ctm_profile_read synchronises the stream and returns, for one class, the
 * timed launches, their summed device time in ms and their algorithmic flop
 * count (2 M N K for a contraction, 0 for Jacobi whose work depends on the
 * data).  When the FP64 class is the only one timed (mask 1), one of its
 * launches in eight is timed.
 * With CTM_PROFILE_SERIAL OR-ed into the mask, moves run eagerly on the
 * context's stream alone (no side streams, no CUDA graphs) until the mask is
 * changed: a calibration mode in which no two kernels of the context overlap, so
 * each class's summed event time is its own device time.
 */
enum { CTM_PROFILE_SERIAL = 0x100 };
int ctm_profile_enable(ctm_ctx* ctx, int on);
int ctm_profile_read(ctm_ctx* ctx, int cls, long long* launches, double* ms, double* flops);

/*
 * Singular values of a device matrix M (row-major rows x cols, device pointer)
 * into the device buffer s (min(rows, cols) doubles), descending and scaled to
 * sum s^2 = 1 -- the same values ctm_corner_spectrum returns for a corner --
 * without allocating any device memory.  (The paper has no counterpart: this
 * serves callers that cannot allocate, e.g. inside a runtime that owns the
 * device memory or forbids cudaMalloc/cudaFree after start-up.)
 * Scratch: one fixed __device__ array inside the library (about 8.1 MB on every
 * GPU that loads it, held until exit) whose device address is looked up during
 * the first call on each device -- make that first call before any stream
 * capture.  Limits: rows * cols <= 1048576 and min(rows, cols) <= 4096, else
 * CTM_ERR_ARG.  All calls share the array: calls whose GPU work overlaps race
 * and must be serialised.  Its cooperative Jacobi launch is ordered with every
 * other cooperative launch of the library on the device (one internal stream
 * per device, joined to `stream` with events), as a context's are.  The call synchronises `stream` (a cudaStream_t) to
 * report CTM_ERR_NOCONV / CTM_ERR_CUDA.  M is not modified.
 */
int ctm_singular_values_noalloc(const double* M, int rows, int cols, double* s,
                                void* stream);

/*
 * Adjoint of the truncated left singular vectors that define a projector (the
 * factorisations of Sec. IV, Fig. 4a, and of the Appendix, differentiated).
 * Inputs, all device memory on the current device, FP64, row-major:
 *   U  rows x r, s r (descending), Vt r x cols -- a thin SVD M = U diag(s) Vt,
 *      r = min(rows, cols);
 *   gU rows x k -- the gradient of a loss with respect to the leading k columns
 *      of U (1 <= k <= r);
 *   eps -- Lorentzian broadening relative to s[0]^4 (e.g. 1e-12; 0 = none).
 * Output gM (rows x cols, caller-allocated):
 *   gM = U [(F o (J - J^T)) diag(s)] Vt + (I - U U^T) gU diag(s_k)^-1 Vt_k,
 *   J = U^T gU (gU zero-padded to r columns), F_ij = E_ij / (E_ij^2 + eps s_0^4),
 *   E_ij = s_j^2 - s_i^2, F_ii = 0 (Liao, Liu, Wang & Xiang 2019; the second
 *   term, Townsend 2016, vanishes when rows <= cols).
 * s and Vt receive no gradient (a projector v v^T uses the left vectors only).
 * Rank-deficient or degenerate input gives a finite gM: with eps = 0 an exactly
 * degenerate pair (s_i = s_j) gets F_ij = 0, and a zero singular value s_j
 * (j < k) gets the pseudo-inverse 0 in diag(s_k)^-1.
 * Stream-ordered on `stream` (a cudaStream_t); temporaries come from the
 * stream-ordered pool; no synchronisation.  Inputs are not modified.
 * Errors: CTM_ERR_ARG (null pointer, k outside [1, r], eps < 0), CTM_ERR_OOM,
 * CTM_ERR_CUDA.
 */
int ctm_svd_left_adjoint(const double* U, const double* s, const double* Vt, const double* gU,
                         int rows, int cols, int k, double eps, double* gM, void* stream);

/*
 * Test hook for the contraction kernels (no counterpart in the paper): C = A B for host row-major A (M x K),
 * B (K x N), C (M x N), computed on the current device in `precision`
 * (CTM_FP64: the FP64 leg-map kernel; CTM_TF32 / CTM_BF16: the tcgen05 kernel
 * with FP32 accumulation).  Allocates its own device buffers; synchronous.
 */
int ctm_contract_test(int precision, long long M, long long N, long long K, const double* A,
                      const double* B, double* C);

/*
 * Test hook for the projector factorisation (no counterpart in the paper; it
 * exposes the truncated SVD that Sec. II-IV and Fig. 4a rely on): U (host,
 * row-major rows x k) receives the leading k left singular vectors of the host
 * row-major matrix M (rows x cols), 1 <= k <= min(rows, cols), computed in FP64
 * on the current device.  path 0 = the library's own choice (exact one-sided
 * Jacobi when min(rows, cols) <= 2048, else the randomized subspace iteration
 * run to convergence), 1 = exact Jacobi, 2 = randomized subspace iteration.
 * k = rows gives the identity.  Columns are sign-fixed (largest-magnitude entry
 * positive) only on the exact path; compare spans, not columns.  Allocates its
 * own device memory; synchronous.  Errors: CTM_ERR_ARG, CTM_ERR_OOM,
 * CTM_ERR_CUDA, CTM_ERR_NOCONV.
 */
int ctm_truncated_svd_test(int path, const double* M, int rows, int cols, int k, double* U);

/*
 * Test hook for the orthonormalisation inside the projector factorisations (no
 * counterpart in the paper; the mixed-precision subspace iteration that stands
 * in for the truncated SVDs of Sec. IV, Fig. 4a, orthonormalises with it):
 * Q (host, row-major rows x n) receives an orthonormal basis of the columns of
 * the host row-major matrix Y (rows x n, n <= rows) from `passes` (1..8) FP64
 * CholeskyQR passes, the first shifted (the library's fused cooperative kernel
 * for n <= 512).  Allocates its own device memory; synchronous.  Errors:
 * CTM_ERR_ARG, CTM_ERR_OOM, CTM_ERR_CUDA.
 */
int ctm_cholqr_test(const double* Y, int rows, int n, int passes, double* Q);

/*
 * Batching of independent states (no counterpart in the paper: many iPEPS
 * states, e.g. of different D and chi, advanced together).  A batch refers to
 * existing contexts (it does not own them; free the batch before them); give
 * each context its own non-default stream so that their work can overlap.
 * ctm_batch_move issues the move of direction dir for every state; once every
 * state is in steady state (bonds at chi, mixed precision, reduced-sequential,
 * caches warm) the moves of all states are captured into one CUDA graph (forked
 * from and joined to a stream the batch owns) and later moves replay it as a
 * single launch.  Results equal those of ctm_move on each context.
 */
typedef struct ctm_batch ctm_batch;
int ctm_batch_create(ctm_batch** out, ctm_ctx** ctxs, int n);
int ctm_batch_move(ctm_batch* batch, int dir, int mode);
const char* ctm_batch_last_error(ctm_batch* batch);
void ctm_batch_free(ctm_batch* batch);

/* Message of the last failure on ctx ("" if none); valid until the next call.
 * (Bookkeeping; no counterpart in the paper.) */
const char* ctm_last_error(ctm_ctx* ctx);

/* Release every device and host resource of ctx (NULL is allowed).
 * (Bookkeeping; no counterpart in the paper.) */
void ctm_free(ctm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* CTM_H */
