/*
 * hap.h - C ABI of the GB300 (sm_103a) Hierarchical Affinity Propagation library.
 *
 * Method: D. M. Rose et al., "Parallel Hierarchical Affinity Propagation with
 * MapReduce" (arXiv:1403.7394), §2 Eqs. 2.1-2.8 and Algorithm 1, iterated with
 * the data-parallel schedule of §3 (every (i, l) of an iteration is updated from
 * the state at the start of that iteration; tau and c are not updated in the
 * first iteration).
 *
 * Conventions shared by every entry point
 *   - Levels are 0-based (the paper's level l is index l-1).  Node i indexes
 *     rows, candidate exemplar j indexes columns (the tensor layout of §3).
 *   - Device pointers are CUDA global-memory addresses of the current device;
 *     host pointers are ordinary CPU memory.  Each argument says which.
 *   - The library never frees memory it did not allocate and keeps no pointer
 *     passed by the caller after the call returns, except the workspace given to
 *     hap_create, which it borrows until hap_destroy.
 *   - All work is enqueued on the stream bound with hap_set_stream (default: the
 *     legacy default stream).  Calls documented as "synchronising" wait for that
 *     stream and report device-side errors; other calls may return before the
 *     GPU work finishes, and an asynchronous fault surfaces at the next
 *     synchronising call as HAP_ECUDA.
 *   - Every function returns HAP_OK (0) or a negative HAP_E* code; no C++
 *     exception or abort crosses this boundary.  hap_strerror names the code.
 *   - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef HAP_H_
#define HAP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define HAP_OK            0
#define HAP_EINVAL       (-1) /* bad argument (null pointer, size, option)          */
#define HAP_ENOMEM       (-2) /* workspace too small / device allocation failed     */
#define HAP_ECUDA        (-3) /* a CUDA runtime call or kernel launch failed        */
#define HAP_EDEVICE      (-4) /* a kernel reported an error in the status word      */
#define HAP_ETIMEOUT     (-5) /* a bounded device-side wait gave up                 */
#define HAP_EUNSUPPORTED (-6) /* valid request this build or device cannot serve    */

/* ---- option values ----------------------------------------------------- */
/* Cluster preference c (Eq. 2.6).  PAPER: c_i^l = max_j(alpha_ij^l + rho_ij^l)
 * every iteration from the second on (§3).  FIXED: c stays at its initial
 * value (0, or hap_set_cluster_preferences), which makes L = 1 flat AP.      */
#define HAP_C_PAPER 0
#define HAP_C_FIXED 1
/* Level schedule.  JACOBI: all levels of an iteration read the state at the
 * start of the iteration (the MR-HAP jobs of §3); neither c nor tau is
 * updated in the first iteration.  GAUSS_SEIDEL: Algorithm 1's sequential
 * level loop - for l = 1..L: rho^l (Eq. 2.1 with the tau^l that level l-1
 * sent in this iteration), then alpha^l (Eqs. 2.2-2.3), then the messages
 * level l sends: c^l (Eq. 2.6, c_mode PAPER), tau^{l+1} (Eq. 2.4) and
 * phi^{l-1} (Eq. 2.5) from the new alpha^l and rho^l; updates from the first
 * iteration on.  Three launches per level and about 32 B moved per message
 * update instead of 17.                                                       */
#define HAP_SCHED_JACOBI       0
#define HAP_SCHED_GAUSS_SEIDEL 1
/* Storage type of the similarity S.                                          */
#define HAP_S_F32  0
#define HAP_S_BF16 1
/* Similarity build (hap_build_similarity), s_ij = -||x_i - x_j||^2 (§2).
 *   F32:        CUDA cores, FP32, direct difference form.
 *   BF16:       tcgen05 tensor cores, x in BF16, FP32 accumulation of x_i.x_j;
 *               norms in FP32 from the FP32 x.
 *   BF16_SPLIT: as BF16 with x = hi + lo split into two BF16 terms and
 *               x_i.x_j ~ hi.hi + hi.lo + lo.hi (three tensor-core products). */
#define HAP_SBUILD_F32        0
#define HAP_SBUILD_BF16       1
#define HAP_SBUILD_BF16_SPLIT 2

/* hap_query keys */
#define HAP_Q_BLOCK_THREADS 1 /* threads per CTA of the row pass              */
#define HAP_Q_CLUSTER_SIZE  2 /* CTAs per cluster (one cluster holds one row)  */
#define HAP_Q_GRID_CLUSTERS 3 /* clusters in the persistent row-pass grid     */
#define HAP_Q_LD            4 /* padded row stride of A, R, S in elements     */
#define HAP_Q_ITER          5 /* completed iterations                          */
#define HAP_Q_ELEMS_PER_THREAD 6 /* columns per thread of the row pass     */
#define HAP_Q_LAUNCHES      7 /* kernels this context has launched so far      */
#define HAP_Q_BATCH_ITEMS_PER_CTA 8 /* batch scheduling granularity (tuned)      */
#define HAP_Q_COL_SUMS      9 /* where the row pass keeps its column sums (HAP_COLSUM_*) */
#define HAP_Q_STAGES       10 /* TMA ring stages of the row pass                */
#define HAP_Q_CTAS_PER_SM  11 /* row-pass CTAs resident per SM (1, or 2 for TMEM
                                 sums with <= 256 threads per CTA)              */

/* Where each row-pass thread keeps the running column sums of max(0, rho) of
 * its columns (Eqs. 2.2-2.4) while its cluster walks its rows.  Both give the
 * same bits for the same grid; they differ in how long a row fits on chip. */
#define HAP_COLSUM_AUTO 0 /* the variant, cluster size and CTAs per SM whose
                             co-resident clusters cover the most SMs with no
                             CTA left without columns, then fewer CTAs per
                             cluster, then one CTA per SM, then TMEM; shared
                             memory when an explicit launch shape is given     */
#define HAP_COLSUM_SMEM 1 /* shared memory: 4, 8 or 16 columns per thread      */
#define HAP_COLSUM_TMEM 2 /* tensor memory (TMEM): 8 or 16 columns per thread,
                             up to 512 threads; frees shared memory for the TMA
                             ring, so a cluster holds twice as long a row      */

typedef struct hap_options {
    int c_mode;        /* HAP_C_PAPER (default) or HAP_C_FIXED                         */
    int schedule;      /* HAP_SCHED_JACOBI (default) or HAP_SCHED_GAUSS_SEIDEL         */
    int s_dtype;       /* HAP_S_F32 (default) or HAP_S_BF16                            */
    int s_per_level;   /* 0 (default): one N x N similarity shared by all levels, the
                          diagonal of level l being the preferences of level l;
                          1: L separate matrices (hap_set_similarity per level)        */
    int block_threads; /* row-pass launch shape, 0 = automatic                         */
    int cluster_size;  /* 0 = automatic; 1..16                                         */
    int grid_clusters; /* 0 = automatic (all co-resident clusters)                     */
    int elems_per_thread; /* 0 = automatic (8); 4, 8 or 16 columns per thread          */
    int profile;       /* 1: time every row-pass launch with CUDA events               */
    int col_sums;      /* HAP_COLSUM_AUTO (default), HAP_COLSUM_SMEM or HAP_COLSUM_TMEM */
    float kappa;       /* Eq. 2.7, the optional level-wise similarity update, read
                          element-wise: s^{l+1}_ij = s^l_ij + kappa (alpha^l_ij +
                          rho^l_ij) for i != j (the printed index j is both free and
                          bound), from the start-of-iteration messages; the
                          diagonal stays the preference of level l+1.  In [0, 1]
                          (the paper's range); 0 (default) = off.  Needs the JACOBI
                          schedule and one S shared by all levels; the net
                          similarity keeps using the given S.                         */
    int64_t wait_limit_ns; /* limit of every bounded device-side wait of the row pass
                          (TMA ring stages, the cluster's row exchange), in
                          nanoseconds; 0 (default) = 2 s.  A wait that runs out
                          makes the kernel stop, let its own copies land and
                          return; the next synchronising call reports
                          HAP_ETIMEOUT.  Minimum 1.                                  */
    int ctas_per_sm;   /* row-pass CTAs per SM: 0 = automatic (1 for an explicit
                          launch shape), 1, or 2 (TMEM column sums, <= 256 threads
                          per CTA: two CTAs share an SM and its tensor memory, so a
                          cluster needs twice the CTAs for a row but clusters can
                          cover more SMs)                                            */
    int debug_bounds;  /* 1: checks for debugging, all reported as HAP_EDEVICE by
                          the next synchronising call (hap_set_similarity and
                          hap_build_similarity: HAP_EINVAL for a non-finite S):
                          every off-diagonal similarity must be finite (§2 admits
                          s_ij = -inf; this library requires finite values); every
                          bulk copy of the row pass must lie inside the messages;
                          the row maximum of Eq. 2.1 must sit in a real column.
                          Failed checks skip the access and never trap.  0 (default)
                          = no checks.                                               */
} hap_options;

typedef struct hap_ctx hap_ctx;

/* Fills *opt with the defaults listed above. */
void hap_default_options(hap_options* opt);

/* Bytes of device workspace hap_create needs for N points and L levels with
 * these options (NULL = defaults).  Host call, no GPU work; fails with
 * HAP_EINVAL for N < 2, L < 1, L > 16 and with HAP_EUNSUPPORTED for N beyond
 * the largest row the row pass holds on chip (65536). */
int hap_workspace_bytes(int64_t N, int L, const hap_options* opt, size_t* bytes);

/* Creates a context for N points and L levels (Algorithm 1 inputs).
 *   prefs        host [L]: preference s_jj of every point at level l (§2), or
 *                NULL for 0; hap_set_preferences gives per-point values.
 *   damping      lambda in (0, 1) (§2): m <- lambda*m_old + (1-lambda)*m_new.
 *   dev_workspace device memory of at least hap_workspace_bytes, 256-byte
 *                aligned, borrowed until hap_destroy; NULL = the context
 *                allocates (cudaMalloc) and frees it itself.
 * The messages start at Algorithm 1's initial values (alpha = rho = 0,
 * tau = +inf, phi = 0, c = 0).  Synchronising. */
int hap_create(int64_t N, int L, const float* prefs, float damping,
               const hap_options* opt, void* dev_workspace, size_t ws_bytes,
               hap_ctx** out);

/* Releases the context (and the workspace if hap_create allocated it). */
void hap_destroy(hap_ctx* ctx);

/* Binds a cudaStream_t (as void*) for all later work of this context. */
int hap_set_stream(hap_ctx* ctx, void* stream);

/* Preferences s_jj^l (§2, the diagonal of S^l).  prefs: host float array,
 * [L] when per_point == 0, [L][N] row-major when per_point == 1.  Takes
 * effect from the next iteration; does not reset the messages. */
int hap_set_preferences(hap_ctx* ctx, const float* prefs, int per_point);

/* Initial / fixed cluster preferences c^l_j (Eq. 2.6's variable; Algorithm 1
 * starts it at 0).  c0: host [L][N] float.  Resets the messages. */
int hap_set_cluster_preferences(hap_ctx* ctx, const float* c0);

/* Copies a similarity matrix into the context and resets the messages to
 * Algorithm 1's initial values.
 *   level  -1: the matrix is used at every level; 0..L-1: only that level
 *          (requires s_per_level = 1).
 *   S      device, N rows of ld elements (ld >= N), row i = node i, column j =
 *          candidate exemplar j; the diagonal is ignored (the preferences are
 *          used instead).  Values must be finite (checked, HAP_EINVAL, with
 *          hap_options.debug_bounds = 1).
 *   dtype  HAP_S_F32 or HAP_S_BF16 (the type of the caller's S); it is
 *          converted to the context's s_dtype (BF16 storage rounds to nearest). */
int hap_set_similarity(hap_ctx* ctx, int level, const void* S, int64_t ld, int dtype);

/* Builds s_ij = -||x_i - x_j||^2 (§2) on the GPU from X and resets the
 * messages.  X: FP32 [N][d] row-major, device memory, or host memory (pinned
 * or pageable): the call then first copies it, on the bound stream, into the
 * message storage it is about to reset, so a host buffer costs no device
 * allocation.  mode: HAP_SBUILD_*.  The result is used at every level.  The
 * tensor-core modes pack their BF16 operands into the message storage, which
 * the workspace sizes for d <= 256; beyond that they may return
 * HAP_EUNSUPPORTED (HAP_SBUILD_F32 has no limit), and so may a host X that does
 * not fit beside the operands (not at N >= 1024).  Synchronising. */
int hap_build_similarity(hap_ctx* ctx, const float* X, int64_t d, int mode);

/* Copies the similarity the iterations use at `level` (0..L-1) into S: device
 * float [N][N] row-major, diagonal = the level's preferences, BF16 storage
 * widened exactly.  Asynchronous. */
int hap_get_similarity(hap_ctx* ctx, int level, float* S);

/* Runs n iterations of HAP (Eqs. 2.1-2.6 with damping, and Eq. 2.7 when
 * kappa > 0) under the context's level schedule on the bound stream.
 * Asynchronous; n >= 0. */
int hap_iterate(hap_ctx* ctx, int n);

/* Eq. 2.8: e_i^l = argmax_j (alpha_ij^l + rho_ij^l), lowest index on ties,
 * from the current messages.  e: int32 [L][N]; on_host = 1: e is host memory
 * and the call is synchronising; 0: e is device memory, asynchronous. */
int hap_exemplars(hap_ctx* ctx, int32_t* e, int on_host);

/* Net similarity NS^l = sum_i s^l_{i, e_i^l} of the current assignment
 * (Eq. 2.8), accumulated in FP64 on the GPU with s^l_ii the preference; the
 * paper does not define an objective, this is the usual AP one.
 * ns: host double [L].  Synchronising. */
int hap_net_similarity(hap_ctx* ctx, double* ns);

/* Acceptance check of the current assignment (Eq. 2.8; the paper prints no
 * convergence test, it runs a fixed count): per level, the number of points
 * whose exemplar is its own exemplar (e_{e_i} = e_i, all N at a
 * self-consistent fixed point) and the number of exemplars (e_i = i).
 * consistent, exemplars: host int64 [L], either may be NULL.  Synchronising. */
int hap_acceptance(hap_ctx* ctx, int64_t* consistent, int64_t* exemplars);

/* Reads the messages after hap_query(HAP_Q_ITER) iterations.
 *   A, R  device float [L][N][N] (alpha, rho), either may be NULL
 *   vecs  device float [3][L][N]: c, tau, phi; may be NULL
 *   iter  host, completed iterations; may be NULL
 * Asynchronous; does not change the context's state. */
int hap_get_state(hap_ctx* ctx, float* A, float* R, float* vecs, int64_t* iter);

/* Replaces the messages (A, R device [L][N][N]; vecs device [3][L][N]: c, tau,
 * phi) and the completed-iteration count, e.g. to resume from a checkpoint.
 * JACOBI uses the c part (tau and phi are recomputed by the next iteration);
 * GAUSS_SEIDEL uses c and phi (phi^l carries the top-down message of the
 * previous iteration).  The next hap_iterate continues exactly as an
 * uninterrupted run would. */
int hap_set_state(hap_ctx* ctx, const float* A, const float* R, const float* vecs, int64_t iter);

/* Waits for the bound stream and checks the device status word.
 * After HAP_ETIMEOUT or HAP_EDEVICE the messages are undefined; the error
 * stays reported until hap_set_state, hap_set_similarity,
 * hap_build_similarity or hap_set_cluster_preferences gives the context a
 * new state (they clear it). */
int hap_sync(hap_ctx* ctx);

/* Changes hap_options.wait_limit_ns of a context (ns >= 1; 0 = 2 s) for the
 * following iterations.  Host call. */
int hap_set_wait_limit(hap_ctx* ctx, int64_t ns);

/* Launch shape and counters (HAP_Q_* keys).  Host call. */
int hap_query(hap_ctx* ctx, int key, int64_t* value);

/* With opt.profile = 1: total milliseconds and number of row-pass launches
 * timed by CUDA events since the last reset (reset = 1 clears after reading).
 * Synchronising. */
int hap_row_pass_time(hap_ctx* ctx, double* ms, int64_t* launches, int reset);

/* ---- batched instances ----------------------------------------------------
 * Many independent HAP problems of uneven N and L advanced together: every
 * iteration is ONE persistent row-pass launch over all instances plus one
 * batched column-statistics launch, replayed from a CUDA graph from the second
 * iteration on.  Instance b has N[b] points (2 <= N[b] <= 4096) and L[b] levels
 * (1..16); rows of small instances are processed up to 16 per step by row
 * groups of one CTA; CTAs claim (instance, band) items largest first from one
 * list, so results do not depend on which CTA ran what.  Same equations and
 * schedule as hap_iterate (data-parallel schedule, kappa = 0).  The context
 * allocates its own device memory (hap_batch_destroy frees it).
 *   N, L   host arrays of B entries.
 * Options used: c_mode, s_dtype, wait_limit_ns (opt may be NULL); another
 * schedule or kappa != 0 gives HAP_EUNSUPPORTED. */
typedef struct hap_batch hap_batch;
int hap_batch_create(int B, const int64_t* N, const int* L, float damping, const hap_options* opt,
                     hap_batch** out);
void hap_batch_destroy(hap_batch* batch);
int hap_batch_set_stream(hap_batch* batch, void* stream);
/* One preference per (instance, level): host float array of sum_b L[b]
 * entries, instance-major. */
int hap_batch_set_preferences(hap_batch* batch, const float* prefs);
/* Builds every instance's s_ij = -||x_i - x_j||^2 from X: device FP32
 * [sum_b N[b]][d], instance-major rows; mode HAP_SBUILD_*.  Resets messages. */
int hap_batch_build_similarity(hap_batch* batch, const float* X, int64_t d, int mode);
/* Copies instance b's similarity (device, N[b] rows of ld elements, dtype
 * HAP_S_*).  Resets the messages of every instance. */
int hap_batch_set_similarity(hap_batch* batch, int b, const void* S, int64_t ld, int dtype);
/* n iterations of every instance; asynchronous. */
int hap_batch_iterate(hap_batch* batch, int n);
/* Eq. 2.8 for every instance: int32, instance-major [sum_b L[b] N[b]]
 * ([L[b]][N[b]] per instance); on_host as for hap_exemplars. */
int hap_batch_exemplars(hap_batch* batch, int32_t* e, int on_host);
/* FP64 net similarity per (instance, level): host double [sum_b L[b]].
 * Synchronising; reports device errors. */
int hap_batch_net_similarity(hap_batch* batch, double* ns);
/* Instance b's messages, as hap_get_state (device buffers for N[b], L[b]). */
int hap_batch_get_state(hap_batch* batch, int b, float* A, float* R, float* vecs, int64_t* iter);
/* Autotuner: times one steady-state iteration for every tile width of the
 * row pass (16 columns per thread with 8192-element ring steps, or 8 columns
 * with 4096-element steps in a deeper ring; 16 needs every L[b] <= 8) and
 * every work-split granularity (items per CTA), and keeps the fastest pair;
 * resets the messages to Algorithm 1's start.  best_ms (may be NULL)
 * receives its time; hap_batch_query gives the choice
 * (HAP_Q_ELEMS_PER_THREAD, HAP_Q_BATCH_ITEMS_PER_CTA). */
int hap_batch_tune(hap_batch* batch, double* best_ms);
/* Sets the tile width by hand: elems_per_thread 16 or 8 (16 needs every
 * L[b] <= 8, else HAP_EUNSUPPORTED).  Resets the messages.  Synchronising. */
int hap_batch_set_tile(hap_batch* batch, int elems_per_thread);
int hap_batch_query(hap_batch* batch, int key, int64_t* value);
/* Waits for the bound stream and checks the device status word: every wait
 * of the batched row pass gives up after the wait limit (hap_options.
 * wait_limit_ns at creation, or hap_batch_set_wait_limit) and reports
 * HAP_ETIMEOUT; the messages are then undefined until hap_batch_set_similarity
 * or hap_batch_build_similarity gives the batch a new state (which clears
 * the report). */
int hap_batch_sync(hap_batch* batch);
/* Changes the wait limit (ns >= 1; 0 = 2 s) for the following iterations.
 * Host call. */
int hap_batch_set_wait_limit(hap_batch* batch, int64_t ns);

/* ---- row bands ---------------------------------------------------------------
 * One HAP problem split by rows (§3: MR-HAP keys the responsibility job by
 * node i, so rows are independent given the column statistics, and the
 * availability job keys by exemplar j, so columns need every row's rho).  A
 * band holds rows row0 .. row0 + nrows - 1 of S, alpha and rho for all L
 * levels; only column statistics cross bands, once per iteration:
 *   1. hap_band_rows on every band: the row pass of one iteration (the same
 *      kernels and equations as hap_iterate) over the band's rows, then the
 *      band's exchange buffer xch [4][L][ld] float (device): its rows' part of
 *      P_j = sum_i max(0, rho_ij), i != j (Eqs. 2.2-2.4), and the c (Eq. 2.6),
 *      phi (Eq. 2.5) and rho_jj of the rows it owns (zero elsewhere);
 *   2. the caller gathers every band's buffer, in band order, into one
 *      device array xch_all [P][4][L][ld] (an all-gather between devices, or
 *      plain copies when the bands share a device);
 *   3. hap_band_columns on every band: P_j summed in band order (so every band
 *      gets the same bits), c, phi and rho_jj of column j from the band owning
 *      row j, then b_j and tau's column part for the next iteration.
 * With one band covering all rows this gives the bits of hap_iterate with the
 * same launch shape.  A band context allocates its own device memory.
 *   N       points of the whole problem (2 .. 65536); L levels (1 .. 16)
 *   row0, nrows  the band's rows, 0 <= row0, 1 <= nrows, row0 + nrows <= N
 *   prefs   host [L] preferences, or NULL for 0
 *   damping lambda in (0, 1), as for hap_create
 * The messages start at Algorithm 1's initial values; creation is
 * synchronising.
 * Options: c_mode, s_dtype, launch-shape fields, wait_limit_ns; the level
 * schedule must be JACOBI, kappa 0, s_per_level and debug_bounds 0 (else
 * HAP_EUNSUPPORTED). */
typedef struct hap_band hap_band;
int hap_band_create(int64_t N, int64_t row0, int64_t nrows, int L, const float* prefs, float damping,
                    const hap_options* opt, hap_band** out);
void hap_band_destroy(hap_band* band);
int hap_band_set_stream(hap_band* band, void* stream);
/* Copies the band's rows of the similarity: S device, nrows rows (rows row0..
 * of the problem's S) of ld_src >= N elements, dtype HAP_S_*; the diagonal
 * (column row0 + i of row i) is ignored.  Resets the messages to Algorithm 1's
 * start.  Synchronising. */
int hap_band_set_similarity(hap_band* band, const void* S, int64_t ld_src, int dtype);
/* Floats in one exchange buffer (4 * L * ld). Host call. */
int hap_band_exchange_floats(hap_band* band, int64_t* n);
/* Step 1 of an iteration: the row pass over the band, then its exchange
 * buffer into xch (device float [4][L][ld]).  HAP_EINVAL if the previous
 * iteration's hap_band_columns is missing.  Asynchronous. */
int hap_band_rows(hap_band* band, float* xch);
/* Step 3: column statistics from every band's buffer.  xch_all device float
 * [P][4][L][ld] in band order; bounds host int64 [P + 1]: band r owns rows
 * bounds[r] .. bounds[r+1] - 1 (bounds[0] = 0, bounds[P] = N, increasing, one
 * band being this one); 1 <= P <= 64.  Completes the iteration.  HAP_EINVAL
 * before hap_band_rows of the same iteration.  Asynchronous. */
int hap_band_columns(hap_band* band, const float* xch_all, int P, const int64_t* bounds);
/* The band's messages after hap_band_query(HAP_Q_ITER) iterations: A, R device
 * float [L][nrows][N] (may be NULL); vecs device float [3][L][N]: c, tau, phi
 * as this band holds them (c and phi of every point after hap_band_columns,
 * tau of the band's own rows); iter host (may be NULL).  Asynchronous. */
int hap_band_get_state(hap_band* band, float* A, float* R, float* vecs, int64_t* iter);
/* Eq. 2.8 for the band's rows: e int32 [L][nrows] (global column indices);
 * on_host as for hap_exemplars. */
int hap_band_exemplars(hap_band* band, int32_t* e, int on_host);
/* Waits for the bound stream and checks the device status word. */
int hap_band_sync(hap_band* band);
/* HAP_Q_* keys as for hap_query. Host call. */
int hap_band_query(hap_band* band, int key, int64_t* value);

/* ---- learned candidate proposal and sparse HAP ------------------------------
 * Not in the paper (its method is dense, §2): each row keeps K candidate
 * exemplars so that large N needs N*K messages instead of N^2.  Sparse HAP is
 * exactly HAP on a similarity that is -inf outside the candidate graph.  The
 * candidates come from an exact kNN pool, optionally re-ranked by a small MLP
 * that scores how likely each point is an exemplar from its kNN distances.  */

/* Exact M nearest neighbours of every point by squared Euclidean distance,
 * itself excluded, ties to the lower index.  X device FP32 [N][d] (d <= 64);
 * idx int32 / dist FP32 device [N][M] sorted ascending; 1 <= M <= 128, M < N.
 * Asynchronous on `stream`. */
int hap_knn(const float* X, int64_t N, int64_t d, int M, int32_t* idx, float* dist, void* stream);

/* hap_knn with an explicit method (hap_knn uses HAP_KNN_AUTO):
 *   HAP_KNN_CUDA_CORES    FP32 direct differences for every pair.
 *   HAP_KNN_TENSOR_CORES  first pass on tcgen05 tensor cores with the BF16 hi/lo
 *                         split (x.y ~ hi.hi + hi.lo + lo.hi, error ~2^-16 of the
 *                         norms), keeping the M + 16 smallest per query, then the
 *                         exact FP32 direct-difference distances of those
 *                         candidates and the M nearest by (distance, index) - the
 *                         CUDA-core result whenever the true M nearest are among
 *                         the M + 16 first-pass candidates.  M <= 64; allocates
 *                         stream-ordered scratch; if its bounded waits give up
 *                         (a stalled GPU) every output index is -1.  From N =
 *                         1024 the points are first put in a spatial order
 *                         (nearest of N/128 pivots) so that near candidates are
 *                         scanned first; that changes the speed, not the result.
 *   HAP_KNN_AUTO          tensor cores when N*N >= 16e6 and M <= 64. */
#define HAP_KNN_AUTO          0
#define HAP_KNN_CUDA_CORES    1
#define HAP_KNN_TENSOR_CORES  2
int hap_knn_with(const float* X, int64_t N, int64_t d, int M, int method, int32_t* idx, float* dist, void* stream);

/* M nearest members of a subset for every point: candidates are the points
 * subset[0..Ns) (device int32 global indices, distinct), a point never takes
 * itself;
 * idx holds global indices.  Uses a temporary device buffer of Ns*d floats
 * (stream-ordered allocation).  Otherwise as hap_knn. */
int hap_knn_subset(const float* X, int64_t N, int64_t d, const int32_t* subset, int64_t Ns, int M, int32_t* idx,
                   float* dist, void* stream);
/* Kernels launched so far by this process through the stateless proposal
 * entry points (kNN, features, scores, candidates, MLP). */
int64_t hap_proposal_launches(void);

/* hap_knn_subset with an explicit method (HAP_KNN_*). */
int hap_knn_subset_with(const float* X, int64_t N, int64_t d, const int32_t* subset, int64_t Ns, int M, int method,
                        int32_t* idx, float* dist, void* stream);

/* Indices of the H highest scores (device [N]), lower index first on ties,
 * ordered by decreasing score, into hubs device int32 [H].  Asynchronous. */
int hap_top_scores(const float* score, int64_t N, int64_t H, int32_t* hubs, void* stream);

/* The distinct points among n_e exemplar indices (device int32 e, e.g. the
 * [L][N] output of hap_sparse_exemplars; entries outside [0, N) are
 * ignored), in increasing order, into points (device int32, room for N);
 * their number in *count (host).  Used to refine a candidate graph: every
 * point's nearest exemplars of one sparse solve (hap_knn_subset with these
 * points, then hap_select_hub_candidates) as the hubs of the next solve.
 * Uses a stream-ordered temporary of about 8N bytes.  Synchronising. */
int hap_exemplar_points(const int32_t* e, int64_t n_e, int64_t N, int32_t* points, int64_t* count, void* stream);

/* Candidates per row: the row itself, its K_near nearest (pool [N][Mp]),
 * then its nearest hubs (hubnn [N][Mh], global indices) not already taken,
 * then further pool entries; sorted by index, K <= 64.  Asynchronous. */
int hap_select_hub_candidates(const int32_t* pool, int64_t N, int Mp, const int32_t* hubnn, int Mh, int K, int K_near,
                              int32_t* cand, void* stream);

/* Features f_q(i) = log(dist[i][q]) - mean_i log(dist[i][F-1]), q < F <= 32,
 * from hap_knn distances ([N][M] device) into feats device [N][F].  The
 * subtracted mean is returned in *log_scale (host, may be NULL).
 * Synchronising. */
int hap_knn_features(const float* dist, int64_t N, int M, int F, float* feats, float* log_scale, void* stream);

/* MLP proposal network: logit = W3 . relu(W2^T relu(W1^T f + b1) + b2) + b3,
 * width 128, F inputs.  FP32 master parameters (flat: W1 [F][128], b1 [128],
 * W2 [128][128], b2 [128], W3 [128], b3 [1]), BF16 copies of the weights used
 * by forward and backward with FP32 accumulation.  theta0: host FP32 [P]. */
typedef struct hap_mlp hap_mlp;
int hap_mlp_create(int F, const float* theta0, hap_mlp** out);
void hap_mlp_destroy(hap_mlp* mlp);
int hap_mlp_set_stream(hap_mlp* mlp, void* stream);
int hap_mlp_num_params(hap_mlp* mlp, int64_t* P);
/* FP32 master parameters into host theta [P].  Synchronising. */
int hap_mlp_get_params(hap_mlp* mlp, float* theta);
/* logits device [n] from feats device [n][F].  Asynchronous. */
int hap_mlp_forward(hap_mlp* mlp, const float* feats, int64_t n, float* logits);
/* Gradients of mean_s w_s (softplus(z_s) - y_s z_s), w_s = pos_weight for
 * y_s = 1 else 1, with respect to the FP32 parameters (host [P], may be
 * NULL) and the loss (host, may be NULL).  labels device [n] in {0, 1}. */
int hap_mlp_gradients(hap_mlp* mlp, const float* feats, const float* labels, int64_t n, float pos_weight,
                      float* grads, float* loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on those gradients; the
 * loss before the step goes to *loss (host, may be NULL). */
int hap_mlp_train_step(hap_mlp* mlp, const float* feats, const float* labels, int64_t n, float pos_weight, float lr,
                       float* loss);

/* Candidates per row from a kNN pool ([N][M] device, M <= 128): the row
 * itself, the K_near nearest, and the K - 1 - K_near pool members beyond
 * those with the highest score (device [N], lower pool position on ties);
 * score NULL: the K - 1 nearest.  cand device int32 [N][K], each row sorted
 * by index; K <= 64, M >= K - 1.  Asynchronous. */
int hap_select_candidates(const int32_t* pool, int64_t N, int M, const float* score, int K, int K_near,
                          int32_t* cand, void* stream);

/* Sparse HAP context: N points, L levels, K candidates per row (K <= 64),
 * damping, c_mode (HAP_C_*), one preference per level (host [L], NULL = 0).
 * Allocates its device memory; same equations and schedule as hap_iterate. */
typedef struct hap_sparse hap_sparse;
int hap_sparse_create(int64_t N, int L, int K, const float* prefs, float damping, int c_mode, hap_sparse** out);
void hap_sparse_destroy(hap_sparse* sp);
int hap_sparse_set_stream(hap_sparse* sp, void* stream);
/* host prefs: [L] (per_point 0) or [L][N] (per_point 1). */
int hap_sparse_set_preferences(hap_sparse* sp, const float* prefs, int per_point);
/* Candidate graph (device int32 [N][K], every row sorted, containing the row
 * itself; checked, HAP_EINVAL otherwise) and points (device FP32 [N][d]):
 * s = -||x_i - x_j||^2 on the graph.  X is borrowed until the next call for
 * hap_sparse_net_similarity.  Resets the messages.  Synchronising. */
int hap_sparse_set_candidates(hap_sparse* sp, const int32_t* cand, const float* X, int64_t d);
int hap_sparse_iterate(hap_sparse* sp, int n);
/* Eq. 2.8 over the candidates: int32 [L][N] global exemplar indices. */
int hap_sparse_exemplars(hap_sparse* sp, int32_t* e, int on_host);
/* NS^l = sum_i -||x_i - x_{e_i}||^2 (preference for e_i = i) in FP64 from the
 * points, host double [L].  Synchronising. */
int hap_sparse_net_similarity(hap_sparse* sp, double* ns);
/* alpha, rho device [L][N][K] (entry q of row i is candidate cand[i][q]);
 * vecs device [3][L][N] (c, tau, phi).  Asynchronous. */
int hap_sparse_get_state(hap_sparse* sp, float* A, float* R, float* vecs, int64_t* iter);
/* keys HAP_Q_ITER and HAP_Q_LAUNCHES. */
int hap_sparse_query(hap_sparse* sp, int key, int64_t* value);
/* on = 1: every later iteration records CUDA events around its two launches
 * (the row pass; the column statistics, which also clear the bitmap of
 * positive slots the next iteration fills).  Host call. */
int hap_sparse_set_profile(hap_sparse* sp, int on);
/* Milliseconds spent in those two launches, summed over the profiled
 * iterations since the last reset (ms: host double [2]), and their number.
 * Synchronising. */
int hap_sparse_profile_times(hap_sparse* sp, double* ms, int64_t* iterations, int reset);

/* Net similarity of any assignment from the points: NS^l = sum_i
 * -||x_i - x_{e_i}||^2, preference pref[l][i] (device FP32 [L][N]) when
 * e_i = i; X device [N][d], e device int32 [L][N]; ns host double [L].
 * Synchronising. */
int hap_net_similarity_points(const float* X, int64_t N, int64_t d, int L, const int32_t* e, const float* pref,
                              double* ns, void* stream);

/* Allocation-free iterations on caller-owned messages.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc - for example a plugin inside a host application that owns and
 * pre-partitions all device memory, or a latency-sensitive loop that cannot
 * afford cudaMalloc's implicit device-wide synchronisation.  It runs the same
 * kernels as hap_iterate, but keeps the row pass's scratch (column partials,
 * b, tau's column part, rho_jj, a status word) in one fixed device array of
 * this library, hap_noalloc_scratch_bytes() bytes (about 4.3 MB), which every
 * GPU that loads the library holds until the process exits.
 *
 * Limits: L * ld <= 16384 (for example N = 4096 with L = 4), where
 * ld = N rounded up to a multiple of 32; larger problems return
 * HAP_EUNSUPPORTED.  At most 64 row-pass clusters are used.
 *
 * Arguments (all device memory on the current device unless stated):
 *   S      [N][ld] similarity shared by all levels, FP32 (s_dtype HAP_S_F32)
 *          or BF16 (HAP_S_BF16); columns N..ld-1 must hold finite values and
 *          the diagonal is ignored.
 *   pref   float [L][ld]: preferences s_ii^l (first N of each row used).
 *   A, R   float [L][N][ld] alpha and rho after t0 iterations, in/out; the
 *          call writes -inf into A's columns N..ld-1.  After the call they
 *          hold the messages after t0 + n iterations.
 *   c      float [L][ld] cluster preference (in: the value after t0
 *          iterations, or the initial / fixed c; out: after t0 + n).
 *   tau, phi float [L][ld], out (phi's last level is set to 0).
 *   t0     completed iterations before the call (0 = Algorithm 1's start,
 *          A = R = 0); n iterations are run; stream is a cudaStream_t.
 * The call is synchronising and calls no allocating routine.  The first call
 * on each device looks up the array's device address (once per device, with
 * that device current); make that first call before any stream capture.
 * With CUDA's lazy module loading, that first call may also be what loads
 * this library's device code onto the device, which allocates the array
 * there once; later calls allocate nothing.
 * Every call shares the one array and leaves its contents behind; the call
 * clears what must start at zero.  Calls that overlap on the GPU (other host
 * threads or streams, the same device) race on the array. */
int hap_iterate_noalloc(int64_t N, int L, float damping, int c_mode, const void* S, int s_dtype,
                        const float* pref, float* A, float* R, float* c, float* tau, float* phi,
                        int64_t t0, int n, void* stream);

/* Size in bytes of the fixed scratch array used by hap_iterate_noalloc. */
size_t hap_noalloc_scratch_bytes(void);

/* Name of a status code. */
const char* hap_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* HAP_H_ */
