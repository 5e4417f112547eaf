/*
 * C-ABI of the GB300 (sm_103a) direct-coupling multi-level lattice Boltzmann
 * library: a hierarchy of nested 2:1 refined Cartesian levels advanced with the
 * H-RR collision (Sec. 2 of Astoul et al., arXiv 2004.14887) and the DC2
 * direct-coupling cell-vertex interface with recursive sub-cycling (Sec. 3).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every call returns LBM_OK (0) or a negative LBM_ERR_* code; the handle's
 *   lbm_last_error() then holds a one-line message.  Nothing throws across the ABI.
 * - Arrays are level-local boxes, x fastest: a node (x, y, z) of level l has
 *   index x + n_x (y + n_y z), with n from lbm_query_level.  Velocity arrays are
 *   [D][n_nodes].  Values at nodes strictly inside the next finer patch (the
 *   "hole", class LBM_NODE_HOLE) are ignored on input and written as 0.
 * - Co-located nodes (a coarse node on the outline of a finer patch and the
 *   fine node at the same place) must receive identical (rho, u).
 * - The caller owns every input/output buffer.  With on_device != 0 the
 *   pointers are device pointers (e.g. torch CUDA tensors) used in order on the
 *   handle's stream; with on_device == 0 they are host pointers and the call
 *   synchronises the stream before returning.
 * - The library owns the population, interface and history arrays.  They are
 *   allocated at lbm_create_hierarchy through desc->alloc/desc->free when given
 *   (the Python binding backs them with PyTorch's caching allocator), else
 *   through cudaMalloc/cudaFree, and released by lbm_destroy.
 * - All device work is issued on the stream given at creation (a private
 *   non-blocking stream when NULL) and is stream-ordered.  lbm_advance forks part of
 *   a coarse step onto two internal streams of the handle and joins them back into
 *   that stream before the step ends.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_MAX_LEVELS 4
#define LBM_TILE_CONFIGS 5
#define LBM_IFACE_AUTO 0
#define LBM_IFACE_NODE 1
#define LBM_IFACE_SEGMENT 2
#define LBM_BATCH_PERSISTENT 0
#define LBM_BATCH_PHASES 1

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

enum {
    LBM_OK = 0,
    LBM_ERR_BAD_DESC = -1,  /* malformed hierarchy description */
    LBM_ERR_OOM = -2,       /* an allocation failed */
    LBM_ERR_CUDA = -3,      /* a CUDA runtime call failed */
    LBM_ERR_NEWTON = -4,    /* Newton at a TF node did not converge in 10 iterations */
    LBM_ERR_DIVERGED = -5,  /* NaN or Inf met in a reduction */
    LBM_ERR_TIMEOUT = -6,   /* a bounded device-side wait gave up */
    LBM_ERR_ARG = -8        /* bad argument (level index, null pointer, size) */
};

enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16S = 2 };  /* population storage precision */
enum { LBM_NODE_HOLE = 0, LBM_NODE_BULK = 1, LBM_NODE_TF_PARENT = 2, LBM_NODE_HANGING = 3,
       LBM_NODE_TF_CHILD = 4 };

typedef void *(*lbm_alloc_fn)(size_t bytes, void *ctx);
typedef void (*lbm_free_fn)(void *ptr, void *ctx);

/*
 * Hierarchy description.
 *   lattice     9 (D2Q9, velocities numbered as in the paper's Fig. 1) or 19 (D3Q19,
 *               the paper's groups: rest, 6 axes, 12 face diagonals).
 *   n_levels    1..LBM_MAX_LEVELS; level 0 is the coarsest and periodic on every axis.
 *   coarse_n    level-0 nodes per axis (coarse_n[2] = 1 for D2Q9).
 *   box_lo/hi   for level l >= 1: the refined patch [lo, hi) in level-0 cell units.
 *               A patch has (hi-lo)*2^l + 1 nodes per axis (cell-vertex: its outline
 *               nodes are shared with level l-1), except on an axis it spans
 *               entirely (lo = 0, hi = coarse_n), where it is periodic.  Each patch
 *               keeps >= 4 parent cells from its parent's outline and >= 4 parent
 *               cells per face (Sec. 3 needs a coarse stencil around every TF node
 *               and four TF nodes along every face for the hanging-node stencil).
 *   nu0         kinematic viscosity in level-0 lattice units: tau_0 = 1/2 + 3 nu0
 *               (Eq. linkTauNu), tau_{l+1} = 2 tau_l - 1/2 (Eq. rescTau).
 *   sigma       H-RR hybridisation weight of Eq. (a12_HRR) (0.98 in the paper).
 *   dc_variant  2 = DC2 of Table 1 (coarse data on P and M^f); 1 = DC1 (coarse on M^f only).
 *   storage     LBM_F64 (FP64 storage and arithmetic), LBM_F32 (FP32 storage and
 *               arithmetic), LBM_F16S (IEEE half storing f_i - s_i, FP32 arithmetic,
 *               s_i below).  The equilibrium / non-equilibrium rescalings of Eqs.
 *               (rescff) and (rescfc) are FP64 in every mode; the Newton solve runs
 *               in the arithmetic type.
 *   psi_sign    +1/-1 factor on the cubic-Mach correction psi_i of App. A; -1 makes
 *               the correction cancel the rho u^3 defect with Psi as printed.
 *   use_graphs  nonzero: lbm_advance replays one captured CUDA graph per coarse step.
 *   alloc/free/alloc_ctx  optional device allocator (both or neither).
 *   u_shift     LBM_F16S only: the shift of the stored deviation is the equilibrium
 *               s_i = f_i^eq(1, u_shift) of Eq. (fEq_herm); {0, 0, 0} gives s_i = w_i
 *               (f_i - w_i).  A u_shift near the flow's mean velocity leaves only the
 *               perturbation to half precision.  A saved state must be loaded into a
 *               hierarchy with the same u_shift.  Components below 0.3 in magnitude.
 */
typedef struct {
    int lattice;
    int n_levels;
    int64_t coarse_n[3];
    int64_t box_lo[LBM_MAX_LEVELS][3];
    int64_t box_hi[LBM_MAX_LEVELS][3];
    double nu0;
    double sigma;
    int dc_variant;
    int storage;
    int psi_sign;
    int use_graphs;
    lbm_alloc_fn alloc;
    lbm_free_fn free;
    void *alloc_ctx;
    double u_shift[3];
} lbm_hierarchy_desc;

typedef struct lbm_hierarchy *lbm_h;

/* Builds levels, node classes, interface tables (Sec. 3.2 sets, Table 1 couples,
 * App. B corners) and device arrays.  *out is NULL on failure (message via
 * lbm_create_error()). */
LBM_API int lbm_create_hierarchy(const lbm_hierarchy_desc *desc, void *cuda_stream, lbm_h *out);
LBM_API const char *lbm_create_error(void);

/* The same with staircase refinement interfaces of arbitrary shape (Sec. 4.1.2
 * circular interface, Sec. 4.2.2 inclined interface, App. B convex and concave
 * corners): masks[l] (l >= 1; masks and masks[l] may be NULL = the whole box) holds one
 * byte per cell of level l-1 inside level l's box [box_lo, box_hi) (level-0 cell units
 * times 2^(l-1) cells per axis, x fastest), nonzero where level l refines the cell; the
 * caller owns the masks and may free them after the call.  Node classes follow from the
 * refined cells around each node (a coarse node whose cells are all refined is a hole,
 * one with some refined cells is co-located with a TF node; a fine node touching an
 * unrefined cell lies on the interface) and the population sets from reading R4, as for
 * boxes.  A hanging node interpolates along its odd axis from the first complete set of
 * TF nodes among the centred (-3, -1, 1, 3) and one-sided (-1, 1, 3, 5) / (1, -1, -3, -5)
 * 4-point sets, else linearly from the two TF nodes of its edge.  Restrictions, checked
 * (LBM_ERR_BAD_DESC): D2Q9, masks on the finest level only, on a box that spans no axis,
 * no two refined cells meeting at a corner only.  Probes are not available on a masked
 * hierarchy (LBM_ERR_ARG). */
LBM_API int lbm_create_hierarchy_masked(const lbm_hierarchy_desc *desc, const uint8_t *const *masks,
                                        void *cuda_stream, lbm_h *out);

/* Box size n[3], box origin (level-l node units) off[3], active node count and tau_l. */
LBM_API int lbm_query_level(lbm_h h, int level, int64_t n_out[3], int64_t off_out[3], int64_t *n_active,
                    double *tau_out);
/* Node class (LBM_NODE_*) of every box node of a level; host buffer of n_x n_y n_z bytes. */
LBM_API int lbm_node_class(lbm_h h, int level, uint8_t *cls_out);

/* Sets f_i = f_i^(0)(rho, u) (Eq. fEq_herm) on every active node of the level (the
 * paper's initial state) and resets the step counters; the interface history of
 * this level is seeded with the same state. rho [n], u [D][n], FP64. */
LBM_API int lbm_init_fields(lbm_h h, int level, const double *rho, const double *u, int on_device);

/* Advances the whole hierarchy by n coarse steps: level l takes 2^l steps per
 * coarse step in the order of Sec. 3.5 (asynchronous then synchronous fine
 * sub-steps, recursively). */
LBM_API int lbm_advance(lbm_h h, int64_t n_coarse_steps);

/* Density and velocity (zeroth and first moments of the current post-collision
 * populations) of every box node of a level; hole nodes get 0. rho [n], u [D][n], FP64. */
LBM_API int lbm_get_macros(lbm_h h, int level, double *rho_out, double *u_out, int on_device);
/* Current post-collision populations of a level as FP64, [Q][n] (hole nodes 0). */
LBM_API int lbm_get_pops(lbm_h h, int level, double *f_out, int on_device);

/* FP64 volume-weighted mass and momentum of a level over its active nodes with the
 * dual-cell weights in level-0 cell volumes (outline nodes weigh the part of their
 * cell inside the level): out[0] = mass, out[1..3] = momentum.  Returns
 * LBM_ERR_DIVERGED if a NaN or Inf was met.
 * The NaN flag is sticky: a reduction that meets NaN or Inf records it in the handle's
 * device status word, and the word is cleared only by lbm_check_status.  Until then
 * every later lbm_reduce and lbm_reduce_static on the handle returns LBM_ERR_DIVERGED
 * (out still receives the sums), whichever level was reduced. */
LBM_API int lbm_reduce(lbm_h h, int level, double out[4]);

/* Stream-ordered variant of lbm_reduce, for loops that read a diagnostic after every
 * step without stalling the GPU.  Enqueues the same reduction (same weights, same
 * FP64 sums, bitwise equal to lbm_reduce) and a copy of its 4 doubles into out on the
 * handle's stream, and returns without synchronising.
 *   - on_device = 0: out is page-locked host memory (cudaHostAlloc, cudaHostRegister,
 *     a pinned tensor); pageable memory is rejected with LBM_ERR_ARG.  on_device = 1:
 *     out is device memory of the handle's device.
 *   - out holds the result once the stream has passed the copy (lbm_synchronize or
 *     any synchronising call); the caller owns out and keeps it alive until then.
 *   - NaN or Inf is not reported by the return value: the sums hold it, and the
 *     device status word records it (lbm_check_status returns LBM_ERR_DIVERGED and
 *     clears the word).  The record is sticky: until that lbm_check_status, every
 *     lbm_reduce and lbm_reduce_static on the handle returns LBM_ERR_DIVERGED.
 *   - Calls on one handle are ordered; each writes only its own out. */
LBM_API int lbm_reduce_async(lbm_h h, int level, double *out, int on_device);

/* Allocation-free variant of lbm_reduce (the paper has no counterpart; this is a
 * library service).  For callers that may not allocate device memory once they are
 * running -- for instance a host process whose device heap is entirely handed to
 * its own pool allocator, or a fixed-latency control loop that forbids cudaMalloc
 * after start-up.  The per-block partial sums live in a static device array of
 * LBM_STATIC_REDUCE_PARTIALS x 4 doubles (+4 for the result, about 128 KB) that
 * every GPU loading the library holds until the process exits; the call itself
 * calls no cudaMalloc, cudaFree or allocating library routine.
 *   - Same inputs, output and weights as lbm_reduce; out is a host buffer of 4 doubles.
 *   - Levels with more than LBM_STATIC_REDUCE_PARTIALS x 2048 box nodes are rejected
 *     with LBM_ERR_ARG and a message naming the limit.
 *   - The handle's device (the device current at its creation) must be the current
 *     device; otherwise the call returns LBM_ERR_ARG.  The first call on a device
 *     looks up the array's device address (cudaGetSymbolAddress) and caches it; make
 *     that first call before any stream capture on that device.
 *   - All calls share the one array: calls whose work overlaps on the GPU (two
 *     streams, or two host threads) race and may return wrong sums.  Each call
 *     overwrites every partial it reads, so nothing has to be cleared between calls.
 *   - Synchronises the handle's stream; returns LBM_ERR_DIVERGED on NaN or Inf, and,
 *     like lbm_reduce, whenever the handle's sticky NaN record is set (cleared only by
 *     lbm_check_status). */
#define LBM_STATIC_REDUCE_PARTIALS 4096
LBM_API int lbm_reduce_static(lbm_h h, int level, double out[4]);

/* Probes: density time series at n points xyz[3n] (level-0 node units; z ignored in
 * 2-D), sampled after every coarse step of lbm_advance by (bi/tri)linear interpolation
 * of the zeroth moment over the cell of the finest level that holds the point.  At
 * most `capacity` rows are recorded (later steps are not sampled).  Setting probes
 * resets the recorded rows.  LBM_ERR_ARG if a point lies on no level's active cells.
 * lbm_get_probes writes the rows recorded so far to out[rows][n] (host; may be NULL
 * to query *n_samples) and synchronises the stream. */
LBM_API int lbm_set_probes(lbm_h h, int n, const double *xyz, int64_t capacity);
LBM_API int lbm_get_probes(lbm_h h, double *out, int64_t *n_samples);

/* Checkpoint: the state after a completed coarse step (every level's populations, the
 * interface histories of Eq. (TempInt) and the step counter) as one host buffer.
 * lbm_save_state with buf == NULL returns the size in *len; lbm_load_state restores
 * a state saved from a hierarchy of the same description (checked: lattice, storage,
 * FP16 shift, levels, box sizes), after which lbm_advance continues bit for bit as the
 * saved run would have.  Both synchronise the stream. */
LBM_API int lbm_save_state(lbm_h h, void *buf, size_t *len);
LBM_API int lbm_load_state(lbm_h h, const void *buf, size_t len);

/* Batches of independent hierarchies (cfg. "many hierarchies of uneven sizes"):
 * lbm_create_batch builds n D2Q9 hierarchies with the same storage and level count
 * on one stream; lbm_advance on the batch advances all of them together in ONE
 * cooperative persistent launch per call: every phase of the sub-cycle schedule of
 * Sec. 3.5 (history + Newton, gradients + hanging nodes, bulk) is one grid-stride
 * pass over the work of all members, with a grid barrier between dependent phases.
 * A barrier wait longer than 2 s gives up and the launch ends with LBM_ERR_TIMEOUT
 * (read by lbm_check_status).  lbm_batch_member returns member i's handle, owned by
 * the batch, for lbm_init_fields / lbm_get_macros / lbm_reduce / lbm_query_level;
 * lbm_advance on a member is an error.  Members must be initialised together (the
 * batch advances only when all members are at the same step).  lbm_destroy on the
 * batch destroys its members. */
LBM_API int lbm_create_batch(const lbm_hierarchy_desc *descs, int n, void *cuda_stream, lbm_h *out);
LBM_API int lbm_batch_member(lbm_h batch, int i, lbm_h *member);
/* Launch structure of lbm_advance on a batch (the same phases of Sec. 3.5 in the same
 * order, bitwise the same results): LBM_BATCH_PERSISTENT (the default) runs a coarse
 * step as the one cooperative launch described above; LBM_BATCH_PHASES runs every phase
 * as one ordinary launch with one block per work item of all members (bulk tiles,
 * Newton + history, gradients + hanging nodes), ordered by the stream instead of grid
 * barriers.  lbm_autotune on a batch times both over reps coarse steps of the live
 * state and keeps the faster; it advances the batch by 2 (reps + 1) coarse steps, so
 * initialise the members after it; us_out (optional, 2 entries) receives microseconds
 * per coarse step (persistent, phases).  lbm_batch_get_path returns the structure or
 * LBM_ERR_ARG. */
LBM_API int lbm_batch_set_path(lbm_h batch, int path);
LBM_API int lbm_batch_get_path(lbm_h batch);
/* Runs the batch's grid barrier alone over one block per SM; block skip_block (if >= 0)
 * leaves without arriving, so the other blocks' waits run out after limit_us
 * microseconds: returns LBM_ERR_TIMEOUT then, LBM_OK when skip_block < 0.  The
 * device context stays usable either way.  Synchronises the batch's stream. */
LBM_API int lbm_batch_check_barrier(lbm_h batch, int skip_block, int64_t limit_us);

/* Device status word accumulated by the kernels since the last call (cleared on read):
 * returns LBM_OK, LBM_ERR_TIMEOUT, LBM_ERR_NEWTON or LBM_ERR_DIVERGED.  Synchronises
 * the stream. */
LBM_API int lbm_check_status(lbm_h h);
/* Largest Newton iteration count met since creation. */
LBM_API int lbm_max_newton_iters(lbm_h h);

/* Autotuner for the D2Q9 bulk kernel.  LBM_TILE_CONFIGS tile shapes are compiled
 * (threads x rows per thread): 0 = 32x8 threads x 2 rows, 1 = 32x4 x 4, 2 = 32x8 x 1,
 * 3 = 64x4 x 2, 4 = 32x16 x 1.  lbm_autotune times reps launches of every shape on
 * every level (on the current state, which it leaves unchanged) and keeps the fastest
 * per level; us_out (optional, n_levels x LBM_TILE_CONFIGS) receives the measured
 * microseconds per launch.  For a D3Q19 hierarchy the configurations are instead the
 * z chunking of the z-marching bulk kernel: about 4, 2, 8, 1 or 16 waves of CTAs per
 * launch (cfg 0..4).  Synchronises.  lbm_set_tile_config / lbm_get_tile_config set or
 * read a level's configuration directly (e.g. from a cache of earlier autotune
 * results); changing one drops the captured graphs.  Every configuration computes the
 * same per-node arithmetic: results are bitwise identical.  On a batch, lbm_autotune
 * chooses the batch's launch structure instead (see lbm_batch_set_path). */
LBM_API int lbm_autotune(lbm_h h, int reps, double *us_out);
LBM_API int lbm_set_tile_config(lbm_h h, int level, int cfg);
LBM_API int lbm_get_tile_config(lbm_h h, int level, int *cfg);

/* Thread mapping of the interface kernels (Newton and rescalings of Eqs. (system_fi),
 * (rescff), (rescfc); the history of Eq. (TempInt); the TF gradients of Sec. 3.3; the
 * hanging-node interpolation of Sec. 3.2).  LBM_IFACE_NODE takes one node per thread
 * (throughput, for large interfaces); LBM_IFACE_SEGMENT one 16- (D2Q9) or 32-lane
 * (D3Q19) warp segment per node, one population per lane, with warp-shuffle sums
 * (latency, for small interfaces).  Both evaluate the same formulas; their sums run
 * in a different order, so results agree to rounding, not bitwise.  LBM_IFACE_AUTO,
 * the default, takes NODE for launches of at least 32768 nodes.  Changing the mode
 * drops the captured graphs.  Returns LBM_ERR_ARG for another mode, or for a batch
 * (a batch takes NODE for every member: its phases cover all members' interfaces). */
LBM_API int lbm_set_interface_mapping(lbm_h h, int mode);

/* Test hook of the bounded waits of the D3Q19 bulk kernel (the paper has no counterpart;
 * failure detection of this library).  From the next lbm_advance on, every bulk launch
 * of `level` runs with its device-side wait limit set to limit_us microseconds, and
 * its block (bx, by, bz) of the launch grid (see lbm_query_level and the 32 x 8 column
 * tiling; bz is the z chunk) does not issue the copies of the k-th plane stage of its
 * z march.  That block's wait for them gives up after the limit, records
 * LBM_ERR_TIMEOUT in the status word (read by lbm_check_status), waits for the copies
 * it did issue and returns; the other blocks finish normally and the device context
 * stays usable, but the level's state is then invalid (re-initialise it).  The
 * withheld stage must be one the block loads (a plane of its chunk, or the plane on
 * either side, that is not a hole of the level).  level < 0 turns the hook off.
 * Drops the captured graphs.  Returns LBM_ERR_ARG for a D2Q9 hierarchy, a batch, or
 * arguments out of range (limit_us in [1, 1e7]). */
LBM_API int lbm_debug_withhold_copy(lbm_h h, int level, int bx, int by, int bz, int k, int64_t limit_us);

/* Kernel timing: while enabled, lbm_advance launches eagerly and brackets every
 * bulk collide-and-stream launch with CUDA events on the handle's stream.
 * lbm_timing_read returns, per level, the summed device milliseconds and the
 * launch count since enabling.  ms_out and launches_out hold n_levels entries. */
LBM_API int lbm_timing_enable(lbm_h h, int enable);
LBM_API int lbm_timing_read(lbm_h h, double *ms_out, int64_t *launches_out);

/* Kernel launches issued by lbm_advance so far (every launch counts, graph-replayed or not). */
LBM_API int64_t lbm_launch_count(lbm_h h);

/* Bytes of device memory held by the handle. */
LBM_API int64_t lbm_device_bytes(lbm_h h);

LBM_API int lbm_synchronize(lbm_h h);
LBM_API const char *lbm_last_error(lbm_h h);
LBM_API void lbm_destroy(lbm_h h);

#ifdef __cplusplus
}
#endif
#endif
