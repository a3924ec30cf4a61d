/*
 * fmm_gb300.h -- C ABI of the GB300 (sm_103a) Cartesian-Taylor fast multipole
 * method for point sources of arbitrary order (Pepper & Fangohr, "fmmgen:
 * Automatic Code Generation of Operators for Cartesian Fast Multipole and
 * Barnes-Hut Methods", arXiv:2005.12351).
 *
 * What is computed (paper §2 and §3.2):
 *   N point sources at positions x_j carry source moments S_{j,n}, |n| = s
 *   (s = 0 charge, 1 dipole, 2 quadrupole; §2, the "source multipole"
 *   before Eq. (5)).  Every source is also a target.  For each target i the
 *   library returns
 *       phi_i = sum_{j != i} sum_{|n|=s} S_{j,n} D_n(x_i - x_j),
 *       E_i   = -grad phi_i,
 *   where D_n(R) = grad^n (1/|R|) (kernel of §2, Eq. (1); no 4 pi eps0),
 *   approximated by the Cartesian FMM of §3.2: octree with at most n_crit
 *   particles per leaf, P2M/M2M upward, M2L over the dual-tree interaction
 *   lists accepted by the MAC (r_A + r_B)/R < theta (§3.2, Eq. (13), r =
 *   half the cell side), L2L downward, L2P and the P2P near field.
 *
 * Truncation: multipoles keep s <= |m| <= p+s, locals keep |n| <= p, and
 * M2L keeps the terms with |n| + |m| <= p+s, so the derivative tensors of
 * 1/r are needed up to order p+s.
 *
 * Moment layout and sign convention: moments are S_n exactly as in the
 * paper, in graded-lexicographic order within |n| = s:
 *   s = 0: q                      (phi = q / r)
 *   s = 1: S_100, S_010, S_001    (phi = -S.R / r^3; a physical dipole mu
 *                                  with phi = mu.R / r^3 is passed as S = -mu)
 *   s = 2: S_200, S_110, S_101, S_020, S_011, S_002
 *                                 (a quadrupole tensor Q is S_n = Q_n / n!,
 *                                  i.e. Qxx/2, Qxy, Qxz, Qyy/2, Qyz, Qzz/2)
 *
 * Threading and streams: a tree handle is not thread-safe; use one handle
 * per host thread.  All device work of a handle is issued on the stream
 * given at creation, in order.  Calls return once the work is enqueued and
 * the few host-visible sizes (cell and list counts) have been read, so a
 * call may synchronise the stream internally; outputs are complete when the
 * stream is synchronised.
 *
 * Errors: every call returns an fmm_status; nothing aborts and no kernel
 * traps.  fmm_last_error() gives a message for the last failing call.
 */
#ifndef FMM_GB300_H
#define FMM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fmm_tree fmm_tree;   /* opaque: owns all device state of one system */

typedef enum {
    FMM_OK = 0,
    FMM_EINVAL = -1,    /* bad argument (NULL, size, order, theta, non-finite input) */
    FMM_ENOMEM = -2,    /* device allocation failed                                   */
    FMM_EORDER = -3,    /* p or s outside the supported range                         */
    FMM_ECUDA = -4,     /* a CUDA runtime call failed                                 */
    FMM_ETIMEOUT = -5,  /* a bounded device wait gave up                              */
    FMM_EBUDGET = -6,   /* the handle's device-memory budget would be exceeded        */
    FMM_ESTATE = -7     /* call out of order (e.g. evaluate before set_sources)       */
} fmm_status;

typedef enum {
    FMM_FP64 = 0,       /* every step in FP64                                         */
    FMM_FP32 = 1,       /* mixed: FP32 pair and contraction arithmetic, FP64 elsewhere */
    FMM_3XTF32 = 2      /* mixed: split-precision contraction, FP32 pair arithmetic   */
} fmm_precision;

/* Largest supported total order p + s (derivative tensors up to this order). */
#define FMM_MAX_TOTAL_ORDER 12
/* Largest supported source order s. */
#define FMM_MAX_SOURCE_ORDER 2

/*
 * Create an empty system on CUDA device `device`.
 *   cuda_stream : a cudaStream_t (NULL = the legacy default stream); the
 *                 caller keeps it alive for the handle's lifetime.
 *   max_leaf    : n_crit of §3.2: a cell is split while it holds more than
 *                 max_leaf particles (and its level is below 21).  >= 1.
 *   prec        : arithmetic of the P2P and M2L bulk work (fmm_precision).
 *   mem_budget_bytes : upper bound on the device memory the handle may hold
 *                 (0 = unlimited); exceeding it returns FMM_EBUDGET.
 * On success *out owns the handle; release it with fmm_destroy.
 * Allocation failure: a call of any handle that returns FMM_ENOMEM has lost
 * the buffer it was growing, so the handle drops its tree, lists and every
 * cache derived from them; the handle itself stays valid, evaluate calls
 * return FMM_ESTATE until fmm_set_sources (or _batch, _mixed) succeeds again,
 * and from there on results are those of a fresh handle.  (FMM_EBUDGET
 * refuses before anything is released and keeps the handle's state.)
 * Testing hook: when the environment variable FMM_FAIL_ALLOC holds k >= 1 as
 * the handle is created, the handle's k-th device allocation (counted from
 * this call, which makes two) fails as cudaMalloc would, once.
 */
fmm_status fmm_create_tree(fmm_tree **out, int device, void *cuda_stream, int max_leaf,
                           fmm_precision prec, size_t mem_budget_bytes);

/*
 * Load N sources and build the octree (§3.2): Morton keys at depth 21,
 * a stable radix sort by (key, original index), and the cells (level,
 * range, integer coordinates, geometric centre, half side).
 *   positions : DEVICE pointer, n x 3 doubles, row-major (x, y, z).
 *   moments   : DEVICE pointer, n x T(s) doubles, T(s) = (s+1)(s+2)/2, row-
 *               major, the S_n layout described above.  May be NULL iff n == 0.
 *   n         : number of particles, 0 <= n < 2^31.
 *   source_order : s in {0, 1, 2}.
 * The library copies (and permutes) both arrays into its own buffers, so the
 * caller may free or overwrite them once the stream has passed this call.
 * Non-finite positions give FMM_EINVAL.  Invalidates cached lists.
 * FMM_ETIMEOUT if a bounded wait of the radix sort gave up (the sort then
 * finishes exactly by a slower route, but the call reports the event).
 */
fmm_status fmm_set_sources(fmm_tree *t, const double *positions, const double *moments,
                           int64_t n, int source_order);

/*
 * Sources of several orders per particle (§2: "mixed systems"): every
 * particle carries the moments of each order s_lo..s_hi, e.g. a charge and a
 * dipole (0..1), in one row of ntot(s_hi) - ntot(s_lo - 1) doubles in graded
 * order (S_000, then S_100 S_010 S_001, then S_200 S_110 S_101 S_020 S_011
 * S_002, restricted to the orders present).  The expansion takes the lowest
 * order: multipoles s_lo <= |m| <= p + s_lo, so fmm_evaluate's order p and
 * its limit p + s_lo <= 12 refer to s_lo.  Every other rule is that of
 * fmm_set_sources; fmm_update_moments takes rows of the same width.  The FP64
 * form only: FMM_EORDER on an FMM_FP32 / FMM_3XTF32 handle with s_hi > s_lo,
 * and unless 0 <= s_lo <= s_hi <= 2.  The symmetric P2P (p2p_variant 2, the
 * FP64 default) takes mixed systems, each shell's reverse term with its own
 * parity; variants 0 and 1 both run the two-targets-per-thread kernel.
 */
fmm_status fmm_set_sources_mixed(fmm_tree *t, const double *positions, const double *moments,
                                 int64_t n, int s_lo, int s_hi);

/*
 * Load a batch of `count` independent systems and build one octree per system
 * (a forest): system s owns particles [offsets[s], offsets[s+1]) of the
 * concatenated arrays, has its own root box, and never interacts with
 * another system.  Every later phase runs as one launch over all systems.
 *   positions, moments : DEVICE, concatenated, layouts as for fmm_set_sources.
 *   offsets : HOST int64 [count + 1], offsets[0] = 0, non-decreasing; empty
 *             systems are allowed.
 *   count   : 1 .. 2^24.  All systems share source_order (and, in
 *             fmm_evaluate, p and theta).
 * Outputs of fmm_evaluate are in the concatenated order.  fmm_set_sources is
 * the count = 1 case.
 */
fmm_status fmm_set_sources_batch(fmm_tree *t, const double *positions, const double *moments,
                                 const int64_t *offsets, int count, int source_order);

/*
 * Evaluate the FMM (§3.2 FMM traversal) at order p with opening angle theta.
 *   p      : local expansion order, 0 <= p and p + s <= FMM_MAX_TOTAL_ORDER;
 *            p >= 1 when want_field.
 *   theta  : MAC parameter of Eq. (13), 0 < theta < 1 (checked: it must also
 *            keep accepted offsets within +-2^16 finer half-cells).
 *   potential : DEVICE pointer to n doubles, or NULL when !want_potential.
 *   field     : DEVICE pointer to n x 3 doubles (E = -grad phi), or NULL when
 *               !want_field.
 * Outputs are in the caller's original particle order.  The interaction
 * lists are rebuilt when theta differs from the cached value; the
 * derivative tables when theta or p change.  FMM_ETIMEOUT if a bounded
 * device wait gave up (the radix sort of the lists: result still exact; the
 * tensor-core M2L: outputs NaN).
 * The lists are laid out by target from row positions the traversal hands
 * out, each row then sorted by source on chip (rows up to 8192 sources); a
 * longer row sends both lists through a radix sort of (target, source) keys,
 * with the same result.  The environment variable FMM_ROW_SORT_LIMIT (read
 * at every list build; 2 .. 8192) lowers that row length, to exercise the
 * radix path.
 */
fmm_status fmm_evaluate(fmm_tree *t, int p, double theta, int want_potential, int want_field,
                        double *potential, double *field);

/*
 * Multipolar Barnes-Hut (§2 multipole potential; §3.2 Methods) on the
 * current tree: multipoles of order p (s <= |m| <= p) by P2M at the leaves
 * and M2M upward, then for every particle a walk from its system's root: a
 * cell with r_cell^2 < theta^2 |x_p - x_c|^2 (r_cell = half the cell side,
 * strict) contributes by M2P, phi += sum_m M_m D_m(x_p - x_c) and
 * E -= sum_m M_m D_{m+e_k}(x_p - x_c) (the exact gradient of that sum); a
 * leaf that fails contributes its particles directly (P2P, the particle
 * itself and coincident points excluded); any other cell that fails is
 * opened.  FP64 whatever the handle's precision; theta = 0 opens every cell
 * (the direct sum).  Outputs as fmm_evaluate (device pointers, the caller's
 * order).  FMM_EORDER unless s <= p <= 12; FMM_EINVAL for theta < 0 or not
 * finite.  Replaces the multipole arrays of the handle (copy_array); a
 * captured fmm_evaluate_graph is dropped.
 */
fmm_status fmm_evaluate_bh(fmm_tree *t, int p, double theta, int want_potential, int want_field,
                           double *potential, double *field);

/* Release all device memory of the handle.  NULL is accepted. */
fmm_status fmm_destroy(fmm_tree *t);

/* Static string for a status code. */
const char *fmm_status_string(fmm_status s);

/* Message of the last failing call on this handle ("" if none).  The pointer
 * stays valid until the next call on the handle.  NULL handle: the message of
 * the last failing fmm_create_tree on this host thread. */
const char *fmm_last_error(const fmm_tree *t);

/* ------------------------------------------------------------------------ */
/* Introspection (tests, benchmarks).                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n;              /* particles                                         */
    int64_t ncells;         /* cells, breadth-first (level, Morton prefix) order */
    int64_t nleaves;
    int32_t nlevels;        /* deepest level + 1                                 */
    int32_t source_order;
    int64_t n_m2l;          /* M2L pairs in the cached lists (0 if none)          */
    int64_t n_p2p;          /* P2P leaf pairs in the cached lists                 */
    int64_t n_p2p_interactions; /* sum over P2P pairs of n_target * n_source      */
    int64_t n_doffsets;     /* distinct M2L offsets (rows of the D table)         */
    double theta;           /* theta of the cached lists (0 if none)             */
    double lo[3];           /* root box corner                                   */
    double side;            /* root box side (a power of two)                    */
    int64_t device_bytes;   /* device memory held by the handle                  */
    int64_t nsystems;       /* independent systems (1 after fmm_set_sources)      */
    /* FMM_3XTF32 tensor-core M2L plan of the last evaluate (0 otherwise):
     * target tiles of 128, (tile, key) rows, chunks of rows; the fill
     * n_m2l / (128 tc_rows) is the share of MMA rows that carry a pair */
    int64_t tc_tiles, tc_rows, tc_chunks;
    /* the last fmm_evaluate_bh (0 before one): M2P evaluations (target, cell)
     * and P2P pairs evaluated (target, leaf particle; the target itself
     * included, it contributes zero) */
    int64_t bh_m2p, bh_p2p;
    int64_t source_order_hi; /* highest source order per particle (= source_order */
                             /* unless fmm_set_sources_mixed)                      */
} fmm_tree_info;

fmm_status fmm_get_info(const fmm_tree *t, fmm_tree_info *out);

/* Identifiers for fmm_copy_array.  Element types and counts:
 *   FMM_ARR_KEYS        uint64 [n]   Morton keys in sorted order
 *   FMM_ARR_PERM        int32  [n]   perm[k] = original index of sorted slot k
 *   FMM_ARR_CELL_LEVEL  int32  [ncells]
 *   FMM_ARR_CELL_COORD  int32  [ncells x 3] integer cell coordinates
 *   FMM_ARR_CELL_RANGE  int32  [ncells x 2] sorted-particle range [begin, end)
 *   FMM_ARR_CELL_PARENT int32  [ncells] (-1 for the root)
 *   FMM_ARR_CELL_CHILD  int32  [ncells x 2] (first child or -1, child count)
 *   FMM_ARR_CELL_CENTRE double [ncells x 3]
 *   FMM_ARR_CELL_HALF   double [ncells]   half side
 *   FMM_ARR_M2L         int32  [n_m2l x 2] (target, source), sorted
 *   FMM_ARR_P2P         int32  [n_p2p x 2] (target, source), sorted
 *   FMM_ARR_MULTIPOLE   double [ncells x n_M] M of the last evaluate
 *   FMM_ARR_LOCAL       double [ncells x n_L] L of the last evaluate
 *   FMM_ARR_CELL_SYSTEM int32  [ncells] system (batch index) of each cell
 * In FMM_FP32 and FMM_3XTF32 handles M and L are the scaled FP32 expansions
 * (float [ncells x n_M], float [ncells x n_L]): M~ = M / h^(|m|-s),
 * L~ = L h^(|n|+s+1), h the cell's half side.
 */
typedef enum {
    FMM_ARR_KEYS = 0, FMM_ARR_PERM, FMM_ARR_CELL_LEVEL, FMM_ARR_CELL_COORD,
    FMM_ARR_CELL_RANGE, FMM_ARR_CELL_PARENT, FMM_ARR_CELL_CHILD, FMM_ARR_CELL_CENTRE,
    FMM_ARR_CELL_HALF, FMM_ARR_M2L, FMM_ARR_P2P, FMM_ARR_MULTIPOLE, FMM_ARR_LOCAL,
    FMM_ARR_CELL_SYSTEM
} fmm_array;

/* Copy one internal array into a HOST buffer of `bytes` bytes (synchronous).
 * FMM_EINVAL if the buffer is too small; *written receives the byte count. */
fmm_status fmm_copy_array(const fmm_tree *t, fmm_array which, void *host_dst, size_t bytes,
                          size_t *written);

/* Per-phase device times of the last evaluate (milliseconds, CUDA events on
 * the handle's stream) when profiling is on.  Phases, in order:
 *   0 keys+bbox, 1 sort, 2 cells, 3 lists, 4 D tables, 5 upward pass (P2M
 *   and M2M, one launch), 6 fold of the multipoles for the harmonic M2L,
 *   7 M2L, 8 L2L (all levels, one launch; in the FP32 forms two: the cells
 *   with children, then the leaves with each leaf's L2P, when the tree has
 *   more than one level), 9 L2P (its own launch: the
 *   FP64 form, and one-level trees), 10 P2P (incl. un-permute)
 * Phases 0-2 belong to fmm_set_sources, 3-10 to fmm_evaluate.  In the FP32
 * forms the M2L plan and operator images of new lists are built on a side
 * stream while the upward pass runs; the M2L phase includes any wait for them. */
#define FMM_NUM_PHASES 11
fmm_status fmm_set_profiling(fmm_tree *t, int enable);
fmm_status fmm_get_phase_times(const fmm_tree *t, float *ms_out /* FMM_NUM_PHASES */);

/* Number of kernels this handle has launched since creation. */
int64_t fmm_launch_count(const fmm_tree *t);

/* ------------------------------------------------------------------------ */
/* Reference evaluation on the GPU.                                          */
/* ------------------------------------------------------------------------ */
/*
 * FP64 direct sum (the plain definition above, no tree) at selected targets:
 *   positions/moments : DEVICE, as for fmm_set_sources;
 *   targets   : DEVICE int32 [n_targets] original indices, or NULL for all n;
 *   potential : DEVICE double [n_targets] or NULL; field: DEVICE [n_targets x 3]
 *               or NULL.
 * Enqueued on cuda_stream; no allocation.
 */
fmm_status fmm_direct_sum(void *cuda_stream, const double *positions, const double *moments,
                          int64_t n, int source_order, const int32_t *targets, int64_t n_targets,
                          double *potential, double *field);

/* fmm_direct_sum for sources of the orders s_lo..s_hi per particle (rows as
 * fmm_set_sources_mixed). */
fmm_status fmm_direct_sum_mixed(void *cuda_stream, const double *positions, const double *moments,
                                int64_t n, int s_lo, int s_hi, const int32_t *targets,
                                int64_t n_targets, double *potential, double *field);

/*
 * Morton order of a point set (the first two steps of fmm_set_sources as a
 * standalone call): the root box of fmm_set_sources, 63-bit keys at depth 21,
 * and a stable sort by (key, original index).
 *   positions : DEVICE n x 3 doubles.
 *   keys_out  : DEVICE uint64 [n], keys in sorted order.
 *   perm_out  : DEVICE int32 [n], perm_out[k] = original index of slot k.
 * Allocates its scratch (about 13 bytes per point) with cudaMalloc and frees
 * it before returning; synchronises cuda_stream.  FMM_EINVAL for non-finite
 * positions; FMM_ETIMEOUT if a bounded wait of the radix sort gave up (the
 * result is still exact).
 * The bound of those waits: each look-back of a sort tile reads the word it
 * waits for at most 2^20 times, or as many times as the environment variable
 * FMM_SORT_POLLS says when it is set (read on every sort, by every entry point
 * that sorts); FMM_SORT_POLLS=0 makes every look-back give up at once, so
 * every tile after the first recounts the digits before it (slow, exact) and
 * the call returns FMM_ETIMEOUT -- a way to exercise that recovery path.
 */
fmm_status fmm_morton_order(void *cuda_stream, const double *positions, int64_t n,
                            uint64_t *keys_out, int32_t *perm_out);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of independent evaluation requests.          */
/* ------------------------------------------------------------------------ */
typedef struct fmm_server fmm_server;

/* One evaluation request.  All arrays are HOST memory owned by the caller,
 * who keeps them alive (and does not touch the outputs) until
 * fmm_server_wait returns for the ticket. */
typedef struct {
    const double *positions;  /* n x 3                                       */
    const double *moments;    /* n x T(s), layout as fmm_set_sources          */
    int64_t n;
    int source_order;         /* 0, 1, 2                                      */
    int p;                    /* expansion order, p + s <= 12                 */
    double theta;             /* MAC parameter, 0 < theta < 1                 */
    int max_leaf;             /* n_crit                                       */
    int want_potential, want_field;
    double *potential;        /* n, or NULL                                   */
    double *field;            /* n x 3, or NULL                               */
} fmm_request;

typedef struct {
    int64_t ticket;
    fmm_status status;
    int slot;                 /* worker that ran it                           */
    double submit_s, start_s, end_s;   /* steady-clock seconds               */
    int64_t device_bytes;     /* device memory of the slot after the request  */
    char message[128];        /* error text when status != FMM_OK             */
} fmm_request_result;

typedef struct {
    int64_t completed, failed, queued, running;
    int64_t device_bytes;      /* held + reserved across slots now            */
    int64_t peak_device_bytes;
    int64_t particles_done;
    double busy_span_s;        /* first start to last completion              */
} fmm_server_stats;

/*
 * A server with `slots` workers on `device`.  Each worker owns a CUDA stream
 * and a resident handle (fmm_create_tree with the given precision), so the
 * trees, lists and expansions of the requests it runs stay on the device.
 * Requests are admitted first-in first-out as soon as a worker is idle and
 * the request's estimated device memory, added to what the other workers
 * hold or have reserved, stays within mem_budget_bytes (0 = unlimited);
 * requests admitted while others run overlap on the GPU.  Workers that sit
 * idle release their buffers when the head of the queue does not fit.
 * This is the paper's evaluation (§3.2) served to many clients; the paper
 * itself has no serving layer.
 */
fmm_status fmm_server_create(fmm_server **out, int device, int slots, fmm_precision prec,
                             size_t mem_budget_bytes);
/* Queue a request; *ticket identifies it.  FMM_EBUDGET if it could never fit. */
fmm_status fmm_server_submit(fmm_server *s, const fmm_request *r, int64_t *ticket);
/* *done = 1 once the ticket has completed (successfully or not). */
fmm_status fmm_server_poll(fmm_server *s, int64_t ticket, int *done);
/* Block until the ticket completes; fills *res (may be NULL) and releases the
 * ticket.  Returns the request's own status. */
fmm_status fmm_server_wait(fmm_server *s, int64_t ticket, fmm_request_result *res);
fmm_status fmm_server_get_stats(fmm_server *s, fmm_server_stats *out);
/* Drain the queue, join the workers and free everything. */
fmm_status fmm_server_destroy(fmm_server *s);

/*
 * Repeated evaluation of one geometry.
 *
 * fmm_update_moments replaces the source moments of the current tree (DEVICE,
 * n x T(s), the caller's particle order as in fmm_set_sources) and keeps the
 * tree, the lists and every cache; asynchronous on the handle's stream.
 *
 * fmm_evaluate_graph is fmm_evaluate for a loop that repeats one parameter
 * set (p, theta, flags, output pointers): the first call evaluates normally,
 * then captures the evaluate into a CUDA graph; later calls with the same
 * parameters replay it with one graph launch (every phase of the path, all
 * systems of a batch).  Any other parameter set recaptures.  fmm_set_sources,
 * fmm_set_sources_batch and fmm_autotune drop the graph.  Profiling phase
 * times are not updated by replays.  Errors as fmm_evaluate; FMM_ECUDA if
 * the capture fails.
 */
fmm_status fmm_update_moments(fmm_tree *t, const double *moments);
fmm_status fmm_evaluate_graph(fmm_tree *t, int p, double theta, int want_potential, int want_field,
                              double *potential, double *field);

/*
 * Autotuner: times the handle's kernel variants on its own tree and lists
 * (reps evaluates each, after one warm-up, CUDA events on the handle's
 * stream) and keeps the fastest for later evaluates.  Candidates:
 *   FMM_FP64    P2P with one or two targets per thread (p2p_variant 0, 1),
 *               or each mirrored leaf pair once for both directions (2)
 *   FMM_3XTF32  the tensor-core M2L with 8, 16 or 32 key rows per chunk, or
 *               the tiled SIMT FP32 M2L (m2l_tensor 0); then, with the fastest
 *               of those, the P2P tile of the other shape (p2p_targets 1 or 2)
 *   FMM_FP32    the tiled SIMT FP32 M2L with 8, 16 or 32 key rows per chunk,
 *               or one block per target cell (m2l_tiled 0); then the P2P tile
 *               of the other shape
 * The FP32 forms keep their P2P kernel: the one-way kernel (p2p_variant 1,
 * their default) evaluates the pairs closer than one mean particle spacing of
 * the target leaf in double-float arithmetic, which holds the near field's
 * rounding at the FP64 form's level; their symmetric kernel (2, selectable
 * with fmm_set_tuning) evaluates every pair in FP32 and is not a candidate.
 * Defaults before tuning: p2p_variant 2 (FP64) or 1 (FP32 forms), the
 * tensor-core M2L (FMM_3XTF32), the tiled SIMT M2L (FMM_FP32), 16 rows per
 * chunk, harmonic M2L.
 * The variants compute the same sums in another order: results agree to the
 * form's rounding, not bitwise.  Synchronises the stream.  out may be NULL.
 */
typedef struct {
    int p2p_variant;        /* P2P: 0 one target per thread, 1 two, 2 each       */
                            /* mirrored leaf pair once for both directions (the  */
                            /* FP32 forms: 0 and 1 are their two-target kernel)  */
    int m2l_tensor;         /* FMM_3XTF32: 1 tensor-core M2L, 0 SIMT FP32 M2L   */
    int tc_chunk_rows;      /* key rows summed per chunk of the tensor-core M2L  */
    int candidates;         /* variants timed                                    */
    float ms_per_evaluate;  /* time of the chosen variant                        */
    int m2l_harmonic;       /* SIMT M2L (FP64, FP32, 3xTF32 off the tensor cores)*/
                            /* over the traceless components (§3.1): 1 (default) */
                            /* or the full Cartesian sums: 0                     */
    int p2p_targets;        /* FP32 forms' one-way P2P tile: targets per thread, */
                            /* 2 (default; both share each staged source read)   */
                            /* or 1 (more threads per target, fewer registers)   */
    int m2l_tiled;          /* SIMT FP32 M2L (FMM_FP32; FMM_3XTF32 with          */
                            /* m2l_tensor 0): 1 (default) over the tensor-core   */
                            /* plan's target tiles and key rows (tc_chunk_rows   */
                            /* rows summed per chunk), 0 one block per target    */
                            /* cell                                              */
} fmm_tuning;
fmm_status fmm_autotune(fmm_tree *t, int p, double theta, int want_potential, int want_field,
                        double *potential, double *field, int reps, fmm_tuning *out);

/*
 * Applies a tuning, e.g. one fmm_autotune reported for the same workload on
 * an earlier run, without timing anything: p2p_variant 0, 1 or 2,
 * m2l_tensor 0 or 1, tc_chunk_rows in [1, 64], m2l_harmonic 0 or 1,
 * p2p_targets 1 or 2 (0 in a zero-filled struct also keeps the setting); a
 * negative value keeps the handle's current setting, and candidates and
 * ms_per_evaluate are ignored.  The harmonic M2L contracts only the 2k+1
 * components of degree k with m_z <= 1 of the folded multipole and derives
 * the L_n with n_z >= 2 from the Laplace identity D_{k+2x} + D_{k+2y} +
 * D_{k+2z} = 0: the same sums as the full M2L up to rounding, about half the
 * work at p = 6.
 * Variant 2 (the near field by Newton's third law, §3.1 P2P) keeps per
 * mirrored leaf pair a row of reverse terms for each source particle; where
 * those rows exceed the handle's budget, evaluates take variant 1.  The paper
 * has no counterpart for this call.  FMM_EINVAL for a value out of range or a
 * NULL tuning.
 */
fmm_status fmm_set_tuning(fmm_tree *t, const fmm_tuning *tuning);

/*
 * Self-check of the library's own FP64 reciprocal square root used by the
 * P2P near field (an FP32 rsqrtf seed refined by one third-order
 * Householder step in FP64): writes own[i] = the library's 1/sqrt(x[i]) and
 * ref[i] = CUDA's rsqrt(x[i]) for comparison.  x > 0, normal doubles.
 * All pointers DEVICE, n entries; enqueued on cuda_stream, no allocation.
 */
fmm_status fmm_check_rsqrt(void *cuda_stream, const double *x, int64_t n, double *own,
                           double *ref);

/*
 * Self-check of the tensor-core building blocks of the FMM_3XTF32 M2L
 * (tcgen05.mma kind::tf32, M = 128, 32-byte-swizzled K-major operand tiles,
 * accumulator in tensor memory).  Computes, in one block,
 *     D[i][n] = sum_{kb < nkb, n < kbn[kb]} sum_{k < 8} A[i][8 kb + k] B[n][8 kb + k]
 * for i < 128, n < N, with every A and B value split into two TF32 halves;
 * passes = 1 forms hi.hi only, passes = 3 adds hi.lo + lo.hi (3xTF32).
 * a_tmem != 0 stages A in tensor memory instead of shared memory.
 * A: DEVICE [128 x 8 nkb] FP32 row-major; B: DEVICE [N x 8 nkb]; D: DEVICE
 * [128 x N]; kbn: HOST [nkb], multiples of 16 with kbn[0] = N.
 * 1 <= nkb <= 4, 16 <= N <= 256, N % 16 == 0.  Synchronises the device;
 * FMM_ETIMEOUT if the block's bounded wait for the MMAs gave up.  The paper
 * has no counterpart: this pins the hardware layout the M2L relies on.
 */
fmm_status fmm_check_umma(const float *A, const float *B, float *D, int nkb, int N,
                          const int *kbn, int a_tmem, int passes);

/*
 * fmm_morton_order without any device allocation.  The paper has no
 * counterpart: this serves callers that must not allocate device memory
 * while they call the library -- code running inside a custom allocator or
 * memory-pool callback (an allocation would re-enter it), runtimes that give
 * the library a fixed arena and forbid cudaMalloc/cudaFree because those
 * calls synchronise the device, and latency-critical loops.
 *   Arguments and results are those of fmm_morton_order (DEVICE pointers).
 *   Scratch: a file-scope device array of about 13.6 MB holding room for
 *   FMM_NOALLOC_MAX_POINTS points; every GPU that loads the library holds it
 *   until the process exits.  n > FMM_NOALLOC_MAX_POINTS returns FMM_EBUDGET
 *   and touches nothing; n < 0 or NULL pointers return FMM_EINVAL.
 *   Device: the calling thread's current device.  The first call on each
 *   device does a set-up: the CUDA runtime loads the library's module for
 *   that device (which places the scratch array and may itself allocate),
 *   the array's device address is looked up (cudaGetSymbolAddress) and the
 *   sort's shared-memory limit is raised.  A call with n == 0 does only this
 *   set-up (pointers may then be NULL); make it once per device, before any
 *   stream capture and outside any allocator callback, so that later calls
 *   allocate nothing.
 *   Sharing: all calls on a device use the same array, and each call leaves
 *   its contents behind.  Calls that overlap on the GPU (different streams
 *   or threads without ordering between them) race on it: serialise them.
 *   Synchronises cuda_stream before returning; allocates nothing.
 */
#define FMM_NOALLOC_MAX_POINTS (1 << 20)
fmm_status fmm_morton_order_noalloc(void *cuda_stream, const double *positions, int64_t n,
                                    uint64_t *keys_out, int32_t *perm_out);

#ifdef __cplusplus
}
#endif
#endif /* FMM_GB300_H */
