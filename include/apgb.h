/*
 * apgb.h -- C ABI of the GB300 affinity-propagation library (libapgb.so).
 *
 * Method: Xia, Wu, Zhang, Zhuang, "Local and global approaches of affinity
 * propagation clustering for large scale data": Algorithm 1 (affinity
 * propagation, Section 2, Eq. 1-4), Algorithm 2 (partition AP, Section 3) and
 * Algorithm 3 (landmark AP, Section 4).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Matrices are row-major float32 with a leading dimension ``ld`` counted in
 *    elements.  N x N matrices need ld >= N, ld % 4 == 0 and a 16-byte aligned
 *    base pointer (128-bit row loads).  Columns N..ld-1 are never read as data
 *    and never written.
 *  - Every pointer documented "device" is caller-owned device memory; the
 *    library allocates no device memory of its own.  Scratch comes from the
 *    caller's workspace ``ws`` (device, 256-byte aligned, ``ws_bytes`` long),
 *    whose size the matching *_workspace_size query returns.  The workspace
 *    contents are not preserved between calls.
 *  - ``stream`` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls whose output includes a host struct (ap_result*, a float*
 *    documented "host") synchronise that stream before returning; the others
 *    only enqueue work.
 *  - Return value: 0 = AP_OK, > 0 = a warning with valid outputs, < 0 = an
 *    error (outputs undefined).  No C++ exception crosses this boundary.
 *  - Calls are not thread-safe with respect to one workspace.
 */
#ifndef APGB_H
#define APGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define AP_OK                 0
#define AP_NOT_CONVERGED      1   /* max_iter reached; results are valid      */
#define AP_NO_EXEMPLARS       2   /* no point chose itself; idx = -1          */
#define AP_ERR_INVALID_ARG   -1   /* bad size, pointer, alignment or param    */
#define AP_ERR_CUDA          -2   /* a CUDA runtime call failed               */
#define AP_ERR_WORKSPACE     -3   /* ws is NULL, misaligned or too small      */
#define AP_ERR_TIMEOUT       -4   /* a bounded device-side wait gave up       */
#define AP_ERR_NONFINITE     -5   /* S holds NaN or +-Inf                     */
#define AP_ERR_UNSUPPORTED   -6   /* e.g. the GPU is not sm_103               */
#define AP_ERR_TOO_LARGE     -7   /* n exceeds the fixed built-in scratch of a
                                     no-allocation entry                      */
#define AP_ERR_CAPACITY      -8   /* a result outgrew the capacity its
                                     workspace was sized for                  */

/* ---- options --------------------------------------------------------------- */
#define AP_PREC_FP32   0   /* similarity by a float32 SIMT GEMM                  */
#define AP_PREC_BF16   1   /* similarity by a bf16 tcgen05 GEMM, fp32 accumulate */

#define AP_PREF_MEDIAN 0   /* p = median of the off-diagonal similarities        */
#define AP_PREF_SCALAR 1   /* p = pref[0] for every point (pref: host float*)    */
#define AP_PREF_VECTOR 2   /* p(k) = pref[k] (pref: device float[N])             */

/* Parameters of Algorithm 1.  Section 2: each message is damped as
 * lambda*old + (1-lambda)*new with 0.5 <= lambda < 1 (any value in [0,1) is
 * accepted); Step 4 stops after a fixed number of iterations or once the
 * decisions have been constant for some iterations. */
typedef struct ap_params {
    float   damping;      /* lambda in [0, 1)                                     */
    int32_t max_iter;     /* >= 1                                                 */
    int32_t conv_iter;    /* stop once the exemplar set is non-empty and has been
                             identical for conv_iter consecutive iterations;
                             0 = run exactly max_iter iterations                  */
    int32_t check_every;  /* iterations enqueued between host checks of the
                             device-side stop flag; 0 = automatic                 */
    int32_t flags;        /* AP_FLAG_* bits                                       */
} ap_params;

/* ap_params.flags: bracket every sweep launch with CUDA events on the
 * caller's stream and report their summed duration in ap_result.sweep_ms
 * (the iterations are then enqueued as separate launches). */
#define AP_FLAG_TIME_SWEEP 1
/* ap_params.flags: enqueue iterations as separate kernel launches.  By default
 * each chunk of check_every iterations (m sweep + m column-sum launches, when
 * m >= 4) is one CUDA graph: captured on a library-owned stream the first time
 * a workspace address and launch shape are seen, kept (up to 32 per process),
 * and launched on the caller's stream. */
#define AP_FLAG_NO_GRAPH   2
/* ap_params.flags, pap_run only: Step 4 starts from the block-diagonal R of
 * the sub-problems as well as A' (the paper carries availabilities only, so
 * R = 0 without this flag). */
#define AP_FLAG_PAP_CARRY_R 4
/* ap_params.flags: the caller has already checked this S for NaN/Inf (for
 * example an earlier call on the same S, when a run is resumed in chunks);
 * ap_iterate and ap_iterate_batched skip their own check, which reads S once
 * more (4 bytes per element, a fifth of one iteration's traffic). */
#define AP_FLAG_S_CHECKED 8
/* ap_params.flags, ap_iterate and ap_iterate_batched: a cold start (Eq. 1:
 * R = A = 0) whatever R and A hold on entry; the caller need not clear them.
 * The first sweeps read zeros from the workspace instead of R and A, which
 * are then written as usual. */
#define AP_FLAG_COLD 16

/* Outputs of Algorithm 1 (Section 2): dpsim = sum of the data-point
 * similarities to their exemplars, expref = sum of the exemplars'
 * preferences, netsim = dpsim + expref (= -E(c) of the energy in Section 2). */
typedef struct ap_result {
    int32_t iters;        /* iterations whose messages are returned               */
    int32_t converged;    /* 1 if the conv_iter rule stopped the run              */
    int32_t n_exemplars;
    int32_t status;       /* the call's return value, repeated                    */
    double  dpsim, expref, netsim;
    double  sweep_ms;     /* with AP_FLAG_TIME_SWEEP: summed sweep-kernel time    */
    int32_t sweep_launches; /* sweep-kernel launches that did work               */
    int32_t pad;
} ap_result;

/* ---------------------------------------------------------------------------
 * ap_similarity -- s(i,k) = -||x_i - x_k||^2 (Section 2) and the preferences
 * on the diagonal (Algorithm 1 input p(j)).
 *
 *  X        device float32 [n x ldx], row i = x_i (d features used).
 *  S        device float32 [n x lds] output.
 *  precision AP_PREC_FP32 or AP_PREC_BF16.  Both centre X on its mean first
 *           (distances are translation invariant).  BF16 rounds the centred
 *           features to bf16 and takes the squared norms of the rounded
 *           vectors in fp32, so S is the fp32-accumulated negative squared
 *           distance of the rounded points.  Off-diagonal values are clamped
 *           to <= 0.
 *  pref_mode AP_PREF_*; for AP_PREF_MEDIAN the median of the n(n-1)
 *           off-diagonal entries (mean of the two middle order statistics,
 *           formed in double and rounded to float, when n(n-1) is even).
 *  noise_rel, seed  tie-break noise s <- s + noise_rel*|s|*u(i,k) applied to
 *           every entry after the diagonal is set; u(i,k) in [0,1) is the top
 *           53 bits of splitmix64 output number i*n+k+1 of ``seed``, times
 *           2^-53.  noise_rel = 0 skips the pass.
 *  pref_out host float* (may be NULL): receives the scalar preference used
 *           (NaN for AP_PREF_VECTOR).  The call synchronises ``stream``.
 *  Errors: AP_ERR_TIMEOUT if a bounded wait of the tensor-core kernel gave up.
 * ------------------------------------------------------------------------- */
size_t    ap_similarity_workspace_size(int64_t n, int64_t d);
int32_t   ap_similarity(const float* X, int64_t n, int64_t d, int64_t ldx,
                        float* S, int64_t lds, int32_t precision,
                        int32_t pref_mode, const float* pref,
                        double noise_rel, uint64_t seed, float* pref_out,
                        void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * ap_similarity_batched -- ap_similarity for `count` independent problems
 * with the same feature dimension d, in one call (no counterpart in the
 * paper: a batch of independent Algorithm 1 inputs).
 *
 *  X        device float32; problem b's features are rows X + xoff[b]
 *           (n[b] x d, leading dimension ldx).  xoff, n: host int64[count].
 *  S        device float32; problem b's S at S + soff[b], n[b] x n[b] with
 *           leading dimension lds[b] (soff, lds: host int64[count]).
 *  precision, pref_mode as for ap_similarity (AP_PREF_MEDIAN: each
 *           problem's own off-diagonal median; AP_PREF_SCALAR: host pref[0]
 *           for every problem; AP_PREF_VECTOR is not accepted).  No noise.
 *  pref_out host float[count] (may be NULL): the preference of each problem.
 *  Each stage (column means, centring, median passes, diagonal) is one
 *  launch for every problem of the batch on ``stream``; the Gram products
 *  are launched per problem, round-robin over 4 library-owned streams that
 *  fork from and join back to ``stream`` by events.  The workspace holds
 *  every problem's scratch (its centred copy included, sized for float32).
 *  The stream is synchronised once, at the end.  Results equal ap_similarity
 *  on each problem bit for bit.
 *  Errors: AP_ERR_INVALID_ARG for a bad size or offset; AP_ERR_TIMEOUT as for
 *  ap_similarity.
 * ------------------------------------------------------------------------- */
size_t    ap_similarity_batched_workspace_size(const int64_t* n, int32_t count, int64_t d);
int32_t   ap_similarity_batched(const float* X, const int64_t* xoff, const int64_t* n,
                                int32_t count, int64_t d, int64_t ldx, float* S,
                                const int64_t* soff, const int64_t* lds, int32_t precision,
                                int32_t pref_mode, const float* pref, float* pref_out,
                                void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * ap_preference_median -- the preference used when the paper's experiments
 * "adjust the input preference" to a common value (Section 5): the exact
 * median of the n(n-1) off-diagonal entries of S (the diagonal is ignored;
 * mean of the two middle order statistics in double, rounded to float, when
 * n(n-1) is even).  Exact selection on the float32 bit patterns, 3 passes.
 *
 *  S        device float32 [n x ld], n >= 2.
 *  median   host float* out (required); the call is synchronous.
 * ------------------------------------------------------------------------- */
size_t    ap_preference_median_workspace_size(int64_t n);
int32_t   ap_preference_median(const float* S, int64_t n, int64_t ld, float* median,
                               void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * ap_iterate -- the damped message-passing sweep of Algorithm 1:
 *   Eq. 2  r(i,k) <- s(i,k) - max_{k'!=k} (a(i,k') + s(i,k'))
 *   Eq. 3  a(i,k) <- min(0, r(k,k) + sum_{i' not in {i,k}} max(0, r(i',k)))
 *   Eq. 4  a(k,k) <- sum_{i' != k} max(0, r(i',k))
 * R is damped before A is formed from it.  Decisions (Section 2): point i
 * picks the lowest k maximising a(i,k)+r(i,k); E = {k : pick(k) == k}.
 *
 *  S         device float32 [n x ld], preferences on the diagonal.
 *  R, A      device float32 [n x ld], in/out: the initial messages on entry
 *            (zeros for Eq. 1; A' for Algorithm 2 Step 4), the final ones on
 *            return.
 *  decisions device int32 [n] out (may be NULL): each point's pick after the
 *            last iteration.
 *  out       host ap_result* (may be NULL): iters, converged (dpsim/expref/
 *            netsim are left 0; see ap_exemplars).  The call always
 *            synchronises ``stream`` before returning.
 *  Errors: AP_ERR_NONFINITE if S holds NaN/Inf (checked on the device first);
 *  AP_ERR_UNSUPPORTED if no sweep configuration fits n (a cluster of 16 CTAs
 *  covers a row of at most 16 x 1920 float4, n <= 122880, which at 12 bytes
 *  per element of S, R and A is about 180 GB).
 *  Returns AP_NOT_CONVERGED when conv_iter > 0 and max_iter was reached.
 * ------------------------------------------------------------------------- */
size_t    ap_iterate_workspace_size(int64_t n, int64_t ld);
int32_t   ap_iterate(const float* S, float* R, float* A, int64_t n, int64_t ld,
                     const ap_params* params, int32_t* decisions,
                     ap_result* out, void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * ap_iterate_batched -- Algorithm 1 on `count` independent problems
 * (Algorithm 2 Step 2 runs the k sub-matrices this way).  Problem b is the
 * n[b] x n[b] matrix at element offset offsets[b] of the S, R and A arenas,
 * leading dimension ld[b] (offsets[b] % 4 == 0, ld[b] % 4 == 0, n[b] >= 2).
 * Every problem uses `params`; each stops on its own rule.  The problems are
 * grouped into size classes (n split at 512 x 2^(j/4); a class with little
 * work joins the next larger one); the classes run one after another,
 * each with one sweep launch per iteration whose clusters share the rows of
 * the class's running problems evenly.  offsets, n, ld: host arrays.
 * decisions: device int32 arena of sum(n) entries (problem b's after those of
 * problems < b) or NULL.  out: host array of `count` results; with
 * AP_FLAG_TIME_SWEEP, sweep_ms and sweep_launches are those of the problem's
 * size class.  Synchronous.  Returns the largest per-problem status
 * (AP_NOT_CONVERGED if any problem hit max_iter).
 * ------------------------------------------------------------------------- */
size_t    ap_iterate_batched_workspace_size(const int64_t* n, const int64_t* ld, int32_t count);
int32_t   ap_iterate_batched(const float* S, float* R, float* A, const int64_t* offsets,
                             const int64_t* n, const int64_t* ld, int32_t count,
                             const ap_params* params, int32_t* decisions, ap_result* out,
                             void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * pap_run -- partition affinity propagation, Algorithm 2 (Section 3).
 *  Step 1: k diagonal blocks of the given point order: part_offsets (host,
 *          k+1 entries, 0 = first < ... < last = n) or, when NULL, the
 *          paper's rule m = floor(n/k) for blocks 1..k-1 and n - m(k-1) for
 *          block k.
 *  Step 2: Algorithm 1 on every S_jj (the block of S as it stands, global
 *          preferences on its diagonal), all blocks in one batched run.
 *  Step 3: A' = blockdiag(A_11, ..., A_kk), zeros elsewhere, written to A.
 *  Step 4: Algorithm 1 on the whole S from R = 0 (the paper carries only the
 *          availabilities) and A = A'.
 *  Then the outputs of Algorithm 1 (as ap_exemplars) into idx and out->final.
 *  S device [n x ld]; R, A device [n x ld] outputs (final messages);
 *  idx device int32 [n].  `params` applies to Steps 2 and 4.  Synchronous.
 * ------------------------------------------------------------------------- */
typedef struct pap_result {
    int32_t   k;
    int32_t   sub_iters_max;      /* largest Step-2 iteration count          */
    int64_t   sub_iters_sum;
    int32_t   sub_not_converged;  /* Step-2 runs that reached max_iter       */
    int32_t   pad;
    double    sub_ms, merge_ms, final_ms, exemplars_ms;   /* device time     */
    ap_result final;              /* Step 4 iterations and the outputs       */
} pap_result;
size_t    pap_run_workspace_size(int64_t n, int64_t ld, int32_t k, const int64_t* part_offsets);
int32_t   pap_run(const float* S, int64_t n, int64_t ld, int32_t k, const int64_t* part_offsets,
                  const ap_params* params, float* R, float* A, int32_t* idx, pap_result* out,
                  void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * lap_run -- landmark affinity propagation, Algorithm 3 (Section 4), Steps 1
 * and 2 (nearest-exemplar embedding without the max_distance gate).
 *  Step 1: L landmarks chosen by `mode`:
 *    AP_LANDMARK_UNIFORM  the L points with the smallest splitmix64 keys
 *                         key(i) = output i+1 of `seed` (ties by index),
 *                         i.e. a uniform random sample, in ascending order;
 *    AP_LANDMARK_SCORE    the L largest score[i] (device float[n], ties by
 *                         index), in ascending index order;
 *    AP_LANDMARK_GIVEN    landmarks[0..L) (device int32, distinct indices).
 *  then Algorithm 1 on the landmarks' S (ap_similarity with `precision`,
 *  preference = its off-diagonal median) -> c exemplars.
 *  Step 2: every point i gets idx[i] = the exemplar e minimising
 *  |x_i - e|^2 (bf16 tensor-core GEMM of the centred features, fp32
 *  accumulate, arg-max of 2 x.e - |e|^2 fused, lowest exemplar on ties);
 *  exemplars keep themselves.  dpsim = sum over non-exemplars of
 *  -|x_i - x_idx(i)|^2 and expref = c * preference, in float64.
 *  X device float32 [n x ldx]; idx device int32 [n]; landmarks_out device
 *  int32 [L] or NULL.  Synchronous.
 * ------------------------------------------------------------------------- */
#define AP_LANDMARK_UNIFORM 0
#define AP_LANDMARK_SCORE   1
#define AP_LANDMARK_GIVEN   2
typedef struct lap_result {
    int32_t   n_landmarks, n_exemplars;
    float     pref;                 /* preference of the landmark problem    */
    int32_t   pad;
    double    dpsim, expref, netsim;             /* over all n points       */
    double    select_ms, landmark_ms, assign_ms, netsim_ms;  /* device time */
    ap_result landmark;             /* Algorithm 1 on the landmarks          */
} lap_result;
size_t    lap_run_workspace_size(int64_t n, int64_t d, int64_t n_landmarks);
int32_t   lap_run(const float* X, int64_t n, int64_t d, int64_t ldx, int64_t n_landmarks,
                  int32_t mode, const float* score, const int32_t* landmarks, uint64_t seed,
                  int32_t precision, const ap_params* params, int32_t* idx,
                  int32_t* landmarks_out, lap_result* out, void* ws, size_t ws_bytes,
                  void* stream);

/* ---------------------------------------------------------------------------
 * lap_assign -- Algorithm 3 (Section 4) Step 2 on its own: every point joins
 * its nearest centre, for a given set of centres (no max_distance gate).
 *  X        device float32 [n x ldx], the points.
 *  centres  device int32 [c], distinct point indices of the centres (in any
 *           order; "lowest index" on ties means lowest position in this list).
 *  idx      device int32 [n] out: centres[argmin_j |x_i - x_centres[j]|^2],
 *           computed as argmax_j (2 x_i.e_j - |e_j|^2) by the bf16 tensor-core
 *           GEMM of the mean-centred features with fp32 accumulation (the
 *           arg-max fused into its epilogue, the n x c scores never written);
 *           centres keep themselves.  Up to 1024 centres the -|e_j|^2 term
 *           enters the product as an extra bf16 MMA (an exact three-term
 *           split), beyond that the epilogue subtracts it: the two agree
 *           within the fp32 accumulation bound.  The environment variable
 *           APGB_ASSIGN_NORMS = folded | shared | global forces a form where
 *           it fits (for comparing them; every LAP entry point obeys it).
 *  best     device float [n] out or NULL: that maximum score, on the centred
 *           bf16-rounded features (|x_i|^2 - best is the squared distance).
 *  ws       lap_assign_workspace_size(n, d, c) bytes.  Synchronous.
 * ------------------------------------------------------------------------- */
size_t    lap_assign_workspace_size(int64_t n, int64_t d, int64_t c);
int32_t   lap_assign(const float* X, int64_t n, int64_t d, int64_t ldx, const int32_t* centres,
                     int64_t c, int32_t* idx, float* best, void* ws, size_t ws_bytes,
                     void* stream);

/* ---------------------------------------------------------------------------
 * lap_run_full -- Algorithm 3 (Section 4), Steps 1-4:
 *  Step 1  L uniform landmarks (the L points with the smallest splitmix64 keys
 *          of seed + level, ties by index), Algorithm 1 on their S; the
 *          preference is the off-diagonal median of the first level's landmark
 *          S and is kept at every later level and in Step 3.
 *  Step 2  max_distance(j) = the largest squared distance from a landmark of
 *          class j to its exemplar (from the landmark S); every other point
 *          joins its nearest exemplar's class when its squared distance to it
 *          (bf16-rounded features centred on the level's mean, fp32
 *          accumulation, as in lap_run) is below that class's max_distance.
 *  Step 3  the m points left: Algorithm 1 on them when m <= m0 (one point is
 *          its own exemplar); else Steps 1-3 on them (the next level, up to
 *          max_levels levels; points still left after the last level join
 *          their nearest exemplar in Step 4).  Exemplars of every level merge.
 *  Step 4  (the paper asks for the merged centres and classes to be
 *          refined, with the similarities recomputed, without a procedure)
 *          read as a local search on net similarity (-E(c), Section 2) over
 *          the merged set, for up to refine_rounds rounds (0: reassignment
 *          only).  A round:
 *            a. every point's nearest and second-nearest centre (the
 *               assignment GEMM with a top-2 epilogue);
 *            b. the cost of dropping centre e, delta(e) = sum over its class
 *               of d(i, second) - d(i, nearest); e is a candidate when
 *               delta(e) < -p.  Candidates that are one point's nearest and
 *               second-nearest conflict; of such a pair only the one of
 *               smaller (delta, index) may go.  The unblocked candidates are
 *               dropped and their members move to their second centre;
 *            c. every class moves its centre to the member nearest the class
 *               mean (unrounded features, float64), which minimises the
 *               class's summed squared distance;
 *          until a round changes nothing.  Sums are fixed point, so the
 *          result is bitwise reproducible.  Then every point joins its
 *          nearest exemplar of the final set; exemplars keep themselves.
 *  X          device float32 [n x ldx]; n_landmarks (L) in [2, n]; m0 in
 *             [2, n]; max_levels in [1, AP_LAP_MAX_LEVELS]; refine_rounds >= 0.
 *  idx        device int32[n] out: each point's exemplar.
 *  level_of   device int32[n] out (may be NULL): the level whose Step 2 (or
 *             Step 3's Algorithm 1) settled the point, -1 if none did.
 *  out        host lap_full_result*.  The call synchronises ``stream``.
 *  Errors: AP_NO_EXEMPLARS when the first level's landmarks give none (idx
 *  = -1); AP_ERR_CAPACITY if the merged set outgrows min(n, L*max_levels+m0).
 * ------------------------------------------------------------------------- */
#define AP_LAP_MAX_LEVELS 8
typedef struct lap_full_result {
    int32_t levels;                          /* levels whose Steps 1-2 ran       */
    int32_t n_exemplars;                     /* size of the merged set           */
    float   pref;
    int32_t base_case;                       /* 1: Step 3 ended in Algorithm 1   */
    int32_t unassigned[AP_LAP_MAX_LEVELS];   /* points left by each level's gate */
    int32_t exemplars_at[AP_LAP_MAX_LEVELS + 1];
    float   ms;                              /* device time of the call          */
    double  dpsim, expref, netsim;
    int32_t refine_rounds;                   /* refinement rounds run            */
    int32_t refine_removed;                  /* centres dropped over all rounds  */
    int32_t refine_moved;                    /* centres moved to a class medoid  */
    int32_t pad2;
} lap_full_result;
size_t    lap_run_full_workspace_size(int64_t n, int64_t d, int64_t n_landmarks, int64_t m0,
                                      int32_t max_levels);
int32_t   lap_run_full(const float* X, int64_t n, int64_t d, int64_t ldx, int64_t n_landmarks,
                       int64_t m0, uint64_t seed, int32_t precision, const ap_params* params,
                       int32_t max_levels, int32_t refine_rounds, int32_t* idx, int32_t* level_of,
                       lap_full_result* out, void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * lap_refine -- Algorithm 3 (Section 4) Step 4 on its own: the refinement
 * lap_run_full applies to its merged centres (see there), on a given centre
 * set, for up to `rounds` rounds (0: none), followed by the reassignment of
 * every point to its nearest centre of the final set.
 *  X            device float32 [n x ldx].
 *  centres      device int32 [c]: distinct point indices (any order).
 *  pref         the preference p (< 0 for a meaningful refinement) that
 *               every centre costs in net similarity.
 *  centres_out  device int32 [c] out: the refined set, ascending, in its
 *               first out->n_exemplars entries.
 *  idx          device int32 [n] out: each point's centre.
 *  out          host lap_refine_result*: rounds run, centres dropped and
 *               moved, and dpsim / expref / netsim over all n points
 *               (float64, unrounded features).
 *  ws           lap_refine_workspace_size(n, d, c) bytes.  Synchronous.
 *  AP_ERR_INVALID_ARG for a repeated or out-of-range centre.
 * ------------------------------------------------------------------------- */
typedef struct lap_refine_result {
    int32_t rounds, removed, moved, n_exemplars;
    double  dpsim, expref, netsim;
} lap_refine_result;
size_t    lap_refine_workspace_size(int64_t n, int64_t d, int64_t c);
int32_t   lap_refine(const float* X, int64_t n, int64_t d, int64_t ldx, const int32_t* centres,
                     int64_t c, float pref, int32_t rounds, int32_t* centres_out, int32_t* idx,
                     lap_refine_result* out, void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Learned warm start.  The paper has no learned part: this network plays the
 * role of Algorithm 2's merged availabilities (a warm start for Algorithm 1)
 * and its exemplar score can choose Algorithm 3's landmarks (the non-uniform
 * landmark selection Section 4 leaves to future work).
 *
 * Features of point k (APL_IN = 25), with `scale` > 0 (e.g. |median
 * preference|):
 *   0-15  the 16 largest off-diagonal s(k,j), decreasing (ties: lower j
 *         first), divided by scale;
 *   16-17 mean and standard deviation of the off-diagonal s(k,j), / scale;
 *   18    s(k,k) / scale;
 *   19-22 log(1 + #{j != k : s(k,j) >= -q*scale}), q = 1/8, 1/4, 1/2, 1
 *         (thresholds formed in float32);
 *   23    D(k) - max D(j) over the 16 neighbours j of features 0-15, where
 *         D = feature 20;
 *   24    the fraction of those neighbours with D(j) > D(k).
 * Network 25 -> 256 -> 256 -> 3 with ReLU; outputs (c_hat, a_hat, logit):
 * the predicted converged column value min(0, r(k,k) + a(k,k))/scale (what
 * the warm start writes into column k), a(k,k)/scale and the exemplar
 * log-odds.
 * The input is first standardised, x -> (x - mu) * isd, with mu and isd
 * fixed (set by the caller from training features; their gradient is zero).
 * Parameters: one flat float32 vector of apl_param_count() entries (W1 256x25,
 * b1, W2 256x256, b2, W3 3x256, b3, mu 25, isd 25, row-major), plus a bf16
 * copy (same offsets) that the products use with fp32 accumulation.
 * Training loss (mean over rows): (c_hat - t_c)^2 + (a_hat - t_a)^2 +
 * softplus(logit) - t_e * logit; Adam (0.9, 0.999, 1e-8, bias-corrected).
 * All device pointers are caller-owned; rows-sized scratch comes from `ws`
 * (apl_workspace_size(rows) bytes).  The calls below enqueue work only.
 * ------------------------------------------------------------------------- */
#define APL_IN  25
#define APL_HID 256
#define APL_OUT 3
int64_t   apl_param_count(void);
/* F: device float [n x 25] out.  ws: apl_features_workspace_size(n) bytes
 * (the neighbour lists between the two passes). */
size_t    apl_features_workspace_size(int64_t n);
int32_t   apl_features(const float* S, int64_t n, int64_t ld, float scale, float* F /*n x 25*/,
                       void* ws, size_t ws_bytes, void* stream);
int32_t   apl_targets(const float* R, const float* A, const int32_t* decisions, int64_t n,
                      int64_t ld, float scale, float* T /*n x 3*/, void* stream);
size_t    apl_workspace_size(int64_t rows);
int32_t   apl_sync_bf16(const float* P, void* P16, void* stream);
int32_t   apl_forward(const float* P, const void* P16, const float* F, int64_t rows,
                      float* Y /*rows x 3*/, void* ws, size_t ws_bytes, void* stream);
/* One Adam step on a batch: forward, loss (device float, may be NULL),
 * backward, update of P, M, V (moments) and the bf16 copy.  step >= 1.
 * grad (device float[apl_param_count()] or NULL) receives the gradient. */
int32_t   apl_train_step(float* P, void* P16, float* M, float* V, int64_t step, float lr,
                         const float* F, const float* T, int64_t rows, float* loss, float* grad,
                         void* ws, size_t ws_bytes, void* stream);
/* R <- 0; A <- the column-constant availabilities of the predictions: at a
 * fixed point of Eq. 3-4, a(k,k) = colp(k) and a(i,k) = min(0, r(k,k) +
 * colp(k)) up to the i-th term, so A(i,k) = min(0, c_hat_k * scale) for
 * i != k and A(k,k) = max(0, a_hat_k * scale). */
int32_t   apl_warm_start(const float* Y, int64_t n, float scale, float* R, float* A, int64_t ld,
                         void* stream);

/* apl_warm_start_batched: features, forward pass and warm start of every
 * problem of a batch in one call.  Problem b's S, R and A are n[b] x n[b]
 * (row stride ld[b]) at element offset offsets[b] of the arenas S, R, A;
 * scale: host float[count] (each problem's |preference|).  R <- 0 and A <-
 * the column-constant availabilities of apl_warm_start, per problem.  Y:
 * device float [sum n x 3] out (the predictions, problem after problem) or
 * NULL.  ws: apl_warm_start_batched_workspace_size(n, count) bytes.
 * Features are those of apl_features bit for bit; enqueues work only. */
size_t    apl_warm_start_batched_workspace_size(const int64_t* n, int32_t count);
int32_t   apl_warm_start_batched(const float* S, float* R, float* A, const int64_t* offsets,
                                 const int64_t* n, const int64_t* ld, int32_t count,
                                 const float* scale, const float* P, const void* P16, float* Y,
                                 void* ws, size_t ws_bytes, void* stream);
/* The network's input standardisation from training features F [rows x 25]:
 * mu = column means, isd = 1 / max(population std, 1e-3), written into P's
 * mu / isd slots (float64 sums in a fixed order).  Enqueues work only. */
int32_t   apl_set_standardisation(float* P, const float* F, int64_t rows, void* stream);
/* The judge (host only): use_warm[b] = 1 when |warm - cold| <= tol |cold|
 * (both finite), else 0.  Returns the number of warm results kept. */
int32_t   apl_judge(const double* cold_netsim, const double* warm_netsim, int32_t count,
                    double tol, int32_t* use_warm);

/* apl_ap_run: features -> network -> warm start -> Algorithm 1 -> outputs.
 * With judge != 0 it also runs Algorithm 1 from R = A = 0 (the method without
 * the network) and keeps the warm result only if its net similarity is within
 * 0.5 % of the cold one; otherwise R, A, idx and out->result are the cold
 * run's.  Synchronous. */
typedef struct apl_result {
    int32_t   used_warm;
    int32_t   warm_iters, cold_iters;
    int32_t   pad;
    double    warm_netsim, cold_netsim;
    double    features_ms, forward_ms, warm_ms, cold_ms;   /* device time    */
    ap_result result;
} apl_result;
size_t    apl_ap_run_workspace_size(int64_t n, int64_t ld);
int32_t   apl_ap_run(const float* S, int64_t n, int64_t ld, const float* P, const void* P16,
                     float scale, const ap_params* params, int32_t judge, float* R, float* A,
                     int32_t* idx, apl_result* out, void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Row shards: Algorithm 1 (Section 2) with the rows of S, R and A split
 * between devices (the O(N^2) cost per iteration that Section 3 states is
 * divided by the shard count).  Given the column vectors colp(k) = sum over
 * i' != k of max(0, r(i',k)) and r(k,k), both halves of an iteration are
 * row-local (Eq. 2 needs row i only; Eq. 3-4 need row i, colp and r(k,k)),
 * so each shard sweeps its own rows and the shards exchange, once per
 * iteration, their shares of those two vectors and of the decision counts:
 *
 *   ap_shard_begin                     once
 *   repeat:
 *     ap_shard_sweep(..., red)         one fused sweep over the shard's rows;
 *                                      red <- its shares
 *     red <- sum of red over shards    (the caller's all-reduce: 2n+2 floats)
 *     ap_shard_finish(..., red, &done) c = r(k,k) + colp; stop rule
 *   until done
 *
 * Every shard applies the stop rule to the same totals, so all stop
 * together.  One shard holding every row is Algorithm 1 on one device.
 *  S, R, A     device float32: the shard's rows r0 .. r1-1 of the n x n
 *              matrices, (r1 - r0) x ld each, row j holding global row r0+j
 *              (ld >= n, ld % 4 == 0, 16-byte aligned).  R, A: the initial
 *              messages in, the final ones out (as ap_iterate).
 *  decisions   device int32 [r1 - r0] out or NULL: each row's decision.
 *  red         device float [2n + 2]: (colp share [n], r(k,k) share [n] --
 *              zero off the shard's rows --, exemplar-set changes, exemplars);
 *              ap_shard_sweep writes it, the caller replaces it by its sum
 *              over the shards, ap_shard_finish reads it.
 *  done        host: 1 once the run has stopped; then R holds the final
 *              responsibilities and out (host, may be NULL) iters/converged.
 *  ws          ap_shard_workspace_size(n, ld, r0, r1) bytes, kept across the
 *              calls of one run (it holds the iteration state).  The same
 *              leading arguments go to all three calls.
 *  ap_shard_begin checks the shard's rows for NaN/Inf (AP_ERR_NONFINITE) and
 *  synchronises; ap_shard_sweep only enqueues; ap_shard_finish synchronises.
 * ------------------------------------------------------------------------- */
size_t    ap_shard_workspace_size(int64_t n, int64_t ld, int64_t r0, int64_t r1);
int32_t   ap_shard_begin(const float* S, float* R, float* A, int64_t n, int64_t ld, int64_t r0,
                         int64_t r1, const ap_params* params, int32_t* decisions, void* ws,
                         size_t ws_bytes, void* stream);
int32_t   ap_shard_sweep(const float* S, float* R, float* A, int64_t n, int64_t ld, int64_t r0,
                         int64_t r1, const ap_params* params, int32_t* decisions, float* red,
                         void* ws, size_t ws_bytes, void* stream);
int32_t   ap_shard_finish(const float* S, float* R, float* A, int64_t n, int64_t ld, int64_t r0,
                          int64_t r1, const ap_params* params, int32_t* decisions, const float* red,
                          int32_t* done, ap_result* out, void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Launch configuration of the ap_iterate sweep, and its autotuner.
 *
 * A cluster of `cluster` CTAs spans one row; each CTA owns a slice of the
 * columns, `ept` float4 columns per thread, and stages `stages` rows of its
 * slices of S, R and A in shared memory.  ap_sweep_get_config reports what
 * ap_iterate would use for n points (a pinned configuration, else the
 * built-in heuristic); ap_sweep_set_config pins one for n (NULL unpins).
 * Re-query ap_iterate_workspace_size after pinning: the workspace depends on
 * the configuration.
 *
 * ap_sweep_autotune times every admissible configuration for `iters`
 * fixed iterations on the caller's S (R and A are overwritten: they are
 * tuning scratch), pins the fastest for n and returns it.  Its workspace must
 * hold ap_sweep_autotune_workspace_size(n, ld) bytes.  Synchronous.
 * ------------------------------------------------------------------------- */
typedef struct ap_sweep_config {
    int32_t cluster;    /* CTAs per cluster, 1 .. 16                             */
    int32_t ept;        /* 1..4                                                  */
    int32_t stages;     /* 2..4                                                  */
    int32_t threads;    /* out: threads per CTA                                  */
    int32_t clusters;   /* out: resident clusters launched                       */
    int32_t smem_bytes; /* out: dynamic shared memory per CTA                    */
    float   ms_per_iter;/* out (autotune only): measured time per iteration     */
    int32_t pad;
} ap_sweep_config;
int32_t   ap_sweep_get_config(int64_t n, ap_sweep_config* out);
int32_t   ap_sweep_set_config(int64_t n, const ap_sweep_config* cfg);
size_t    ap_sweep_autotune_workspace_size(int64_t n, int64_t ld);
int32_t   ap_sweep_autotune(const float* S, float* R, float* A, int64_t n, int64_t ld,
                            float damping, int32_t iters, ap_sweep_config* best,
                            void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Work distribution of ap_iterate / ap_iterate_batched, for inspection.
 * Host only: no device is touched.
 *
 * ap_sweep_plan -- the work list a sweep launch uses when problems of sizes
 * n[0..count-1] are all running, with clusters of `cluster` CTAs of which
 * `resident` fit the GPU at once.  Unit u covers rows first, first + stride,
 * ... (count rows) of one problem and owns that problem's column-partial
 * slot; it is written to units[5u .. 5u+4] as (problem, slot, first, count,
 * stride).  Cluster c runs units ubeg[c] .. ubeg[c+1]-1.  units holds cap
 * quintuples (at most resident + count - 1 are needed), ubeg resident + 1
 * entries.  *n_units, *n_clusters: out.  AP_ERR_INVALID_ARG for sizes < 2,
 * cluster outside {1,2,4,8,16}, resident < 1; AP_ERR_WORKSPACE if cap is too
 * small.
 *
 * ap_sweep_classes -- the size class of each problem of a batch (classes
 * are run one after another, each with its own launch configuration):
 * class_of[b] in 0 .. classes-1, in increasing order of size.  Returns the
 * number of classes, or AP_ERR_INVALID_ARG.
 * ------------------------------------------------------------------------- */
int32_t   ap_sweep_plan(const int64_t* n, int32_t count, int32_t cluster, int32_t resident,
                        int32_t* units, int32_t cap, int32_t* ubeg, int32_t* n_units,
                        int32_t* n_clusters);
int32_t   ap_sweep_classes(const int64_t* n, int32_t count, int32_t* class_of);

/* ---------------------------------------------------------------------------
 * ap_exemplars -- outputs of Algorithm 1 from final messages.
 * E = {k : argmax_j (a(k,j)+r(k,j)) == k} (lowest index on ties); exemplars
 * keep idx(k) = k, every other point takes the exemplar of highest s(i,k)
 * (lowest index on ties).  dpsim, expref and netsim are reduced in float64 in
 * a fixed order (bitwise reproducible).
 *
 *  idx   device int32 [n] out; all -1 (and AP_NO_EXEMPLARS) when E is empty.
 *  out   host ap_result* (required): n_exemplars, dpsim, expref, netsim.
 * ------------------------------------------------------------------------- */
size_t    ap_exemplars_workspace_size(int64_t n);
int32_t   ap_exemplars(const float* S, const float* R, const float* A,
                       int64_t n, int64_t ld, int32_t* idx, ap_result* out,
                       void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * ap_exemplars_noalloc -- the same computation and outputs as ap_exemplars,
 * for callers that cannot allocate device memory: plain C callers that only
 * hold pointers into buffers someone else handed them, callers whose device
 * memory is entirely reserved by another framework's caching pool, and code
 * on latency-critical paths where a cudaMalloc would synchronise the device.
 * The paper has no counterpart; this entry exists for deployment only.
 *
 * Instead of a workspace it uses a scratch array built into the library
 * (a file-scope __device__ array of AP_NOALLOC_SCRATCH_BYTES bytes, which
 * every GPU that loads the library keeps until the process exits), so it
 * accepts n <= AP_NOALLOC_MAX_N and returns AP_ERR_TOO_LARGE otherwise.  It
 * calls no cudaMalloc, cudaFree or other allocating routine.  The caller
 * still passes S, R, A, idx and out.
 *  - The first call on each device does the set-up: with that device current
 *    it looks up the array's device address (cudaGetSymbolAddress) and keeps
 *    it for every later call on the device.  Make that first call before any
 *    stream capture begins.  The kept address is never looked up again, so
 *    it does not survive cudaDeviceReset or any other teardown of the
 *    device's primary context: do not call this entry after one in the same
 *    process.
 *  - Like ap_exemplars it fills the host struct `out`, so it returns only
 *    after `stream` has finished the call's work.
 *  - Every call shares the one array, which keeps the previous call's
 *    contents; nothing in it needs to start at zero (every scratch word is
 *    written before it is read).  Calls whose GPU work overlaps (different
 *    streams, different host threads) race on the array: serialise them.
 * ------------------------------------------------------------------------- */
#define AP_NOALLOC_MAX_N         65536
#define AP_NOALLOC_SCRATCH_BYTES (2u << 20)
int32_t   ap_exemplars_noalloc(const float* S, const float* R, const float* A,
                               int64_t n, int64_t ld, int32_t* idx, ap_result* out,
                               void* stream);

/* ---- misc ------------------------------------------------------------------ */
const char* ap_status_string(int32_t status);
int32_t     ap_version(void);            /* major*10000 + minor*100 + patch   */
/* Failure-detection self-test (no counterpart in the paper): one CTA waits on
 * an mbarrier that nothing completes, with the bounded try-wait loop every
 * device wait of the library uses (spin_limit tries).  Returns
 * AP_ERR_TIMEOUT when the bound runs out, as it always should; the context
 * stays usable.  Synchronises ``stream``. */
int32_t     ap_wait_selftest(uint32_t spin_limit, void* stream);
/* Number of kernels this library has launched in this process (all devices,
 * all threads); for accounting in benchmarks. */
uint64_t    ap_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* APGB_H */
