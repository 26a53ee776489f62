/*
 * pma.h - C ABI of the GB300 Voronoi particle-merging library.
 *
 * The library implements the per-cell recursive phase-space partition and
 * merge of Luu, Tueckmantel & Pukhov, "Voronoi particle merging algorithm for
 * PIC codes" (arXiv:1504.00636), Sec. 3 "Algorithm", Steps 1-7:
 *   - Input (Sec. 3): per-particle weight w, position x (dx components) and
 *     momentum p (dp components), tolerances T_X, T_P and N_min; a cell is
 *     merged only when it holds more than N_min particles.
 *   - Step 1: the particles of each simulation cell form the first set V0.
 *   - Step 2: weighted centroid and standard deviation per axis; CVs
 *     Delta_x = sigma/L (Eq. cv_x, L = grid-cell size on that axis) and
 *     Delta_p = sigma/|P| (Eq. cv_p).
 *   - Step 3: a set is final when every Delta is <= its tolerance.
 *   - Step 4 (Eq. step_4): otherwise the axis k with the largest Delta is cut.
 *   - Step 5: V1 = {q_k <= Q_k}, V2 = {q_k > Q_k}.
 *   - Step 6: recurse on V1 and V2.
 *   - Step 7: every final set is replaced by its centroid (W, X, P); a
 *     one-particle set is kept as it is.
 * Output order is canonical: cells ascending, and within a cell the final
 * sets in V1-before-V2 depth-first order.
 *
 * All pointers named "device" are CUDA device pointers (or managed memory)
 * of the current device; "host" pointers are ordinary host memory.  Arrays
 * are structure-of-arrays: pos[a] is the a-th position component of all n
 * particles.  Every function returns a status code (PMA_OK = 0).
 * A handle is not thread-safe: use one handle per host thread / stream.
 */
#ifndef PMA_H
#define PMA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define PMA_OK 0
#define PMA_ERR_INVALID_ARG 1 /* null pointer, bad size, tol < 0 or non-finite */
#define PMA_ERR_INPUT 2       /* particle data: cell id out of range, w <= 0,
                                 non-finite w / x / p (found on the device) */
#define PMA_ERR_CUDA 3        /* a CUDA runtime call failed; see pma_last_error */
#define PMA_ERR_NOMEM 4       /* device or host allocation failed */
#define PMA_ERR_CAPACITY 5    /* n larger than the handle's capacity */
#define PMA_ERR_TIMEOUT 6     /* a bounded device wait gave up (no hang) */
#define PMA_ERR_INTERNAL 7    /* an internal bound was exceeded (reported, not trapped) */

/* ---- precision ------------------------------------------------------- */
#define PMA_FP64 0  /* FP64 storage, plain FP64 sums and decisions */
#define PMA_MIXED 1 /* FP32 storage of x, p, w; compensated FP32 moment sums;
                       FP64 split decision and FP64 merged W and P */

/* ---- config flags ---------------------------------------------------- */
#define PMA_FLAG_NO_INDEX 1u  /* do not accept an output index (saves 4 B/particle) */
/*
 * Decision variants.  Off by default: the default is the paper's rule as
 * printed (Step 4 takes the largest raw Delta_l; Eq. cv_p divides by |P_l|).
 *   PMA_FLAG_SPLIT_NORMALIZED  Step 4 takes the axis of the largest
 *       Delta_l / T_l (T_l = T_X on position axes, T_P on momentum axes; with
 *       T_l = 0 the ratio is +inf when Delta_l > 0 and 0 when Delta_l = 0).
 *   PMA_FLAG_MOMENTUM_NORM  Eq. cv_p uses the length of the mean momentum
 *       vector: Delta_l = sigma_l / |P|, |P| = sqrt(sum over momentum axes
 *       of P_l^2), instead of sigma_l / |P_l|.  Sets whose mean momentum is
 *       near zero on one axis then stop splitting on that axis.
 * They apply to pma_merge and pma_merge_host; pma_merge_noalloc refuses them.
 */
#define PMA_FLAG_SPLIT_NORMALIZED 2u
#define PMA_FLAG_MOMENTUM_NORM 4u
/*
 * Energy-conserving replacement (Step 7 variant; the paper names the idea
 * of merging into two particles in its remark on energy, Sec. 3, without a
 * rule; this rule follows from the conservation laws).  A final set of
 * m >= 3 particles with weight W, centroid X, P and total energy
 * E = sum w sqrt(1 + |p|^2) (p in units of m c) becomes two particles of
 * weight W/2 at X with momenta P + d and P - d, |P +- d|^2 = g^2 - 1,
 * g = E / W: d is orthogonal to P with |d|^2 = g^2 - 1 - |P|^2 (>= 0 by
 * convexity), along the momentum axis e_k of largest sigma_k^2 (1 - Phat_k^2)
 * made orthogonal to P (the axis of smallest |P_k| if all are 0).  With one
 * momentum axis d is along P: d^2 = g^2 (g^2 - 1 - P^2) / (g^2 - P^2).  Sets
 * of two particles are copied as they are, the lower input index first.
 * W, W P and E are conserved to rounding.  out->index maps the members of a
 * set to its first output (a copied pair: each member to its own).  The
 * output count M is still <= n.
 */
#define PMA_FLAG_CONSERVE_ENERGY 8u
/*
 * Energy accounting (Sec. 3, remark on energy: the centroid merge does not
 * keep the energy; the paper measures the loss as delta E = |E0 - E| / E0).
 * With this flag every call also sums the kinetic energy
 * E = sum w (sqrt(1 + |p|^2) - 1) (p in units of m c) of its input and of
 * its output in FP64 (pma_stats.energy_in / energy_out).  It costs an FP64
 * square root per particle, so it is off by default.
 */
#define PMA_FLAG_ENERGY_STATS 16u

typedef struct pma_handle pma_handle;

typedef struct pma_config {
    int32_t dx;           /* position components, 1..3 */
    int32_t dp;           /* momentum components, 1..3 */
    double cell_size[3];  /* L per position axis (Eq. cv_x), > 0 */
    int64_t n_cells;      /* cell ids lie in [0, n_cells); >= 1 */
    int32_t n_min;        /* a cell is merged only if it holds > n_min particles */
    int32_t precision;    /* PMA_FP64 or PMA_MIXED */
    int64_t capacity;     /* largest n of any call; sizes the workspace; <= 2^31-1 */
    uint32_t flags;       /* PMA_FLAG_* */
} pma_config;

/*
 * Near-tie bits of a cell (pma_output.cell_flags).  In exact arithmetic the
 * partition of Steps 2-6 is unique; in floating point a decision taken
 * within rounding of the opposite outcome may differ between two correct
 * implementations.  A cell carries:
 *   PMA_NEAR_STOP    some Delta_l within about 1e-9 (relative) of its
 *                    tolerance in a Step 3 stop test
 *   PMA_NEAR_ARGMAX  the runner-up axis of a Step 4 choice within about 1e-9
 *                    (relative) of the chosen one
 *   PMA_NEAR_CUT     a particle within 64 m eps (|s_k| + sigma_k) of the
 *                    Step 5 cut value Q_k of a set of m particles
 *   PMA_RECHECKED    (PMA_MIXED) an FP32 decision or cut closer than its
 *                    error bound was taken again in FP64 from the particles;
 *                    informational, the result is the FP64 decision
 * With PMA_MIXED every decision is certified: an FP32 comparison is used
 * only when its error bound shows it equals the exact one, so a cell without
 * PMA_NEAR_* bits has the exact-arithmetic partition of its stored values.
 */
#define PMA_NEAR_STOP 1u
#define PMA_NEAR_ARGMAX 2u
#define PMA_NEAR_CUT 4u
#define PMA_RECHECKED 8u

/*
 * Caller-owned device output buffers; every array has room for `capacity`
 * entries (the output count M never exceeds the input count n).
 *   cell[M]           int32 cell id of each merged particle
 *   pos[a][M]         FP64 (PMA_FP64) or FP32 (PMA_MIXED) centroid position
 *   mom[a][M]         FP64 centroid momentum
 *   w[M]              FP64 centroid weight
 *   index[n]          int32: output slot of every input particle, or NULL
 *   count_dev         int64 device word receiving M, or NULL
 *   cell_flags[n_cells]  uint32 PMA_NEAR_* / PMA_RECHECKED bits of every
 *                     cell, or NULL (pma_merge only; the other entry points
 *                     ignore it)
 */
typedef struct pma_output {
    int32_t *cell;
    void *pos[3];
    double *mom[3];
    double *w;
    int32_t *index;
    int64_t *count_dev;
    uint32_t *cell_flags;
} pma_output;

/* Per-call counters (filled after a synchronous call). */
typedef struct pma_stats {
    int64_t n_in;              /* particles in */
    int64_t n_out;             /* merged particles out (M) */
    int64_t cells_merged;      /* cells with more than max(n_min, 1) particles */
    int64_t cells_passthrough; /* cells copied verbatim (1..n_min particles) */
    int64_t splits;            /* Step 4-6 cuts taken */
    int64_t leaves;            /* final sets (Step 7) in merged cells */
    int64_t depth_sum;         /* sum over particles of their final set's depth */
    int64_t degenerate_cuts;   /* cuts whose rounded centroid left a side empty */
    int64_t big_cells;         /* cells too large for one CTA's shared memory */
    int64_t sorted_input;      /* 1 if the cell ids were already non-decreasing */
    int64_t near_stop;         /* decisions flagged PMA_NEAR_STOP */
    int64_t near_argmax;       /* decisions flagged PMA_NEAR_ARGMAX */
    int64_t near_cut;          /* cuts flagged PMA_NEAR_CUT */
    int64_t fp64_rechecks;     /* PMA_MIXED: FP32 decisions taken again in FP64 */
    int64_t cells_flagged;     /* cells with at least one PMA_NEAR_* / PMA_RECHECKED bit */
    int64_t cells_tiny;        /* cells per population path: up to 256 particles */
    int64_t cells_small;       /*   up to the small-class tile (and pass-through) */
    int64_t cells_large;       /*   up to one CTA's shared memory; big_cells above */
    double energy_in;          /* with PMA_FLAG_ENERGY_STATS: kinetic energy in, */
    double energy_out;         /*   and out (summation order varies: last bits) */
} pma_stats;

/*
 * Create a handle: validates cfg, selects the device current at the call,
 * and allocates the device workspace for `capacity` particles.  *out is set
 * on success and untouched on failure.
 */
int pma_create(const pma_config *cfg, pma_handle **out);

/*
 * Merge n particles (Sec. 3, Steps 1-7) on `stream` (a cudaStream_t; 0 =
 * legacy default stream).
 *   cells[n]      device int32 cell id of each particle, in [0, n_cells)
 *   pos[a][n]     device positions, a < dx (FP64 for PMA_FP64, FP32 for PMA_MIXED)
 *   mom[a][n]     device momenta, a < dp (same type)
 *   weights[n]    device weights w > 0 (same type)
 *   tol_x, tol_p  the tolerances T_X, T_P of Step 3, finite and >= 0
 *   out           caller-owned device output buffers (see pma_output)
 *   count_host    host int64 receiving M, or NULL
 * Inputs are never modified.  When count_host is non-NULL the call waits
 * for the stream and returns the status of the device work (PMA_ERR_INPUT
 * for bad particle data); when it is NULL the call only enqueues work and
 * the device status is read by pma_sync().
 */
int pma_merge(pma_handle *h, int64_t n, const int32_t *cells,
              const void *const *pos, const void *const *mom,
              const void *weights, double tol_x, double tol_p,
              const pma_output *out, int64_t *count_host, void *stream);

/*
 * Same as pma_merge with HOST input and output arrays (types as above; the
 * output arrays are host arrays of `capacity` entries).  The handle stages
 * the data through its own device buffers (allocated on first use) and
 * always waits for completion.
 */
int pma_merge_host(pma_handle *h, int64_t n, const int32_t *cells,
                   const void *const *pos, const void *const *mom,
                   const void *weights, double tol_x, double tol_p,
                   const pma_output *out_host, int64_t *count_host, void *stream);

/*
 * Bounded device waits.  The single-pass prefix scans (Step 1 binning and
 * Step 7 output slots) let a CTA wait for the status word of the CTA before
 * it.  Every such wait gives up after `wait_ns` nanoseconds (default 2 s; 0
 * restores it; otherwise >= 1000): the kernel then sets an error bit and
 * returns, the kernels after it in the call return at once, and the call
 * reports PMA_ERR_TIMEOUT.  The device context stays usable and the next
 * call starts afresh.  (No counterpart in the paper: a safeguard of this
 * implementation.)
 */
int pma_set_wait_limit(pma_handle *h, int64_t wait_ns);

/*
 * Bounds-checked build (no counterpart in the paper; it stands in for a
 * memory sanitizer).  A library compiled with -DPMA_CHECKED checks the
 * indices the partition and output kernels use: subset records and tile
 * indices against the shared-memory tile, cut destinations against their
 * subset, final positions and output slots against n, and the cuts of big
 * cells against their cell.  The first index out of range in a call is
 * recorded, its access is skipped, and the call returns PMA_ERR_INTERNAL.
 * pma_checked_build returns 1 for such a library and 0 otherwise.
 * pma_check_first gives the record of the handle's last synchronised call:
 * 0 when every check passed, else (site << 48) | index, the sites numbered
 * 1 subset record, 2 tile index, 3 cut destination, 4 pair record, 5 final
 * position, 6 output slot, 7 big-cell position.  The normal build compiles
 * no checks and always reports 0.
 */
int pma_checked_build(void);
int pma_check_first(const pma_handle *h, uint64_t *site_index);

/*
 * Failure-detection test hook (not for production use; no counterpart in
 * the paper): while `tile` >= 0, every call's Step 1 prefix scan withholds
 * the status word of that scan tile (a tile covers 2048 cells), so that the
 * tile after it waits out its limit and the call returns PMA_ERR_TIMEOUT
 * without faulting or hanging the device.  tile < 0 turns the hook off.
 */
int pma_test_withhold_status(pma_handle *h, int tile);

/*
 * Failure-detection test hook: the status a call reports for a device error
 * word with these bits (1 bad particle data, 4 a bounded wait gave up, 2 an
 * internal bound; the first of these in that order wins, 0 is PMA_OK).
 */
int pma_test_status_of_bits(unsigned bits);

/*
 * Autotuner (no counterpart in the paper, which runs on CPUs: the GPU's
 * choice of which team serves which cells and subsets).  A handle assigns
 * every cell, by its population, to one of four paths, and every pending
 * subset inside a team to one of seven size classes:
 *   caps[0] = cap_t  cells of at most cap_t particles: one-warp teams
 *   caps[1] = cap_w  up to cap_w: 4-warp teams (cap_w <= 1024)
 *   caps[2] = cap    up to cap: 8-warp teams with a tile of cap particles
 *                    (cap <= 8191 and what one CTA's shared memory holds;
 *                    12-warp teams where only one 8-warp CTA fits an SM);
 *                    larger cells are first cut in global memory and their
 *                    pieces join this class
 *   caps[3] = base   the class base B, 12 <= B <= 32: subsets of 3 to B
 *                    particles take one lane each, up to 2B two lanes, ...,
 *                    up to 16B sixteen lanes, larger ones a whole warp (or
 *                    several); pairs have a class of their own
 *   caps[4] = widen  0 or 1: with 1, a round of a size class that has too
 *                    few pending subsets to fill the team gives each subset
 *                    more lanes (up to a warp)
 * with cap_t <= cap_w <= cap.  The result of a merge is the same for every
 * setting (every decision is exact up to the flagged near-ties); only the
 * time differs.  pma_create picks defaults (base 12, widen 0);
 * pma_set_classes sets them (the next call uses them; PMA_ERR_INVALID_ARG when they are out of
 * range) and pma_get_classes reads them.
 *
 * pma_tune times candidate settings on the caller's own particles (the
 * arguments as for pma_merge; at most the first 2^26 particles are used,
 * so the input should be grouped by cell for the prefix to be whole cells):
 * first the population limits with base 12, then the base with the fastest
 * limits, then widen = 1 with the fastest base and with base 24.  It keeps the fastest and synchronises, and writes the outputs as
 * a merge of that prefix would.  When the environment variable
 * PMA_TUNE_CACHE names a file, the choice is looked up there first and
 * stored there afterwards under a key made of D, the precision, the flags,
 * the SM count and the population histogram of the cells (fractions of the
 * particles in cells of 1-64, 65-256, 257-1024, 1025-4096, 4097-8191 and
 * more particles, in twentieths).  The file is a JSON object with one entry
 * per line,
 *   "key": [cap_t, cap_w, cap, base, widen, milliseconds],
 * read and written with pma_tune_cache_lookup / pma_tune_cache_store (host
 * only; lookup returns PMA_ERR_INVALID_ARG when the key is absent).
 */
int pma_get_classes(const pma_handle *h, int32_t caps[5]);
int pma_set_classes(pma_handle *h, const int32_t caps[5]);
int pma_tune(pma_handle *h, int64_t n, const int32_t *cells, const void *const *pos,
             const void *const *mom, const void *weights, double tol_x, double tol_p,
             const pma_output *out, void *stream);
int pma_tune_cache_lookup(const char *path, const char *key, int32_t caps[5]);
int pma_tune_cache_store(const char *path, const char *key, const int32_t caps[5], double ms);

/* Wait for the handle's last enqueued call and return its device status. */
int pma_sync(pma_handle *h);

/* Counters of the last completed call. */
int pma_get_stats(const pma_handle *h, pma_stats *out);

/*
 * Per-stage device timing.  When enabled, every pma_merge records CUDA
 * events on its stream between the stages; pma_get_timing (after the call
 * completed) writes up to n durations in milliseconds, averaged over the
 * calls since timing was enabled (the last 64 of them):
 *   [0] Step 1 binning        [1] big-cell cuts (global memory)
 *   [2] small-cell teams      [3] large-cell teams      [4] big-cell pieces
 *   [5] Step 7 emit           [6] whole call
 * and returns PMA_ERR_INVALID_ARG when timing is off or nothing was timed.
 */
#define PMA_N_STAGES 7
int pma_set_timing(pma_handle *h, int enable);
int pma_get_timing(const pma_handle *h, float *ms, int n);

/*
 * Allocation-free merge.  The paper has no counterpart: this entry point
 * exists for callers that must not allocate device memory, for example a
 * PIC code whose device memory is owned by its own pool allocator, or a
 * host thread that must not trigger the implicit device synchronisation
 * that cudaMalloc/cudaFree can cause in the middle of a time step.  It
 * needs no handle: its scratch is a fixed array inside the library (under
 * 1 MB, held by every GPU that loads the library until the process exits),
 * and the caller passes only inputs and outputs.
 *   cfg          dx, dp, cell_size, n_cells, n_min and precision as for
 *                pma_create; capacity is ignored; flags may hold only
 *                PMA_FLAG_NO_INDEX (the paper's rule and plain Step 7 only:
 *                any other flag returns PMA_ERR_INVALID_ARG)
 *   n, cells, pos, mom, weights, tol_x, tol_p   as for pma_merge; the cell
 *                ids must be non-decreasing (particles grouped by cell)
 *   out          caller-owned device outputs as for pma_merge
 *   count_host   host int64 receiving M, or NULL
 * Limits: n <= PMA_NOALLOC_MAX_N and n_cells <= PMA_NOALLOC_MAX_CELLS,
 * else PMA_ERR_CAPACITY before any device work; every cell with more than
 * n_min particles must fit one CTA's shared memory (over 2,000 particles
 * for D <= 4), else the call returns PMA_ERR_CAPACITY after the device work.
 * Unsorted or out-of-range cell ids and bad particle values return
 * PMA_ERR_INPUT.
 * The call waits for `stream` (it synchronises and copies its status to the
 * host) and returns the device status: it must never be called while its
 * stream is being captured into a CUDA graph.  The first call on each device
 * also looks up the scratch array's device address (once per device, with
 * that device current).  All calls share the one scratch array, which keeps
 * the last call's contents (the part that must start at zero is cleared by
 * every call): calls that overlap on the GPU, from several streams or host
 * threads, race and give wrong results.
 */
#define PMA_NOALLOC_MAX_N 65536
#define PMA_NOALLOC_MAX_CELLS 65536
int pma_merge_noalloc(const pma_config *cfg, int64_t n, const int32_t *cells,
                      const void *const *pos, const void *const *mom,
                      const void *weights, double tol_x, double tol_p,
                      const pma_output *out, int64_t *count_host, void *stream);

/*
 * Measured compute ceiling (no counterpart in the paper; used to place the
 * partition kernels on a roofline): the rate of independent fused
 * multiply-adds per second on the current device in FP32 (PMA_MIXED) or
 * FP64 (PMA_FP64), best of five timed launches over every SM, and the SM
 * count.  Allocates a small device buffer; synchronous.
 */
int pma_probe_fma(int precision, double *fma_per_s, int *sm_count);

/* Release the handle and its device memory (NULL is accepted). */
int pma_destroy(pma_handle *h);

/* Static description of a status code. */
const char *pma_error_string(int code);

/* Text of the last error on this handle ("" if none). */
const char *pma_last_error(const pma_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* PMA_H */
