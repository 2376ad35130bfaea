/*
 * acs.h - C ABI of the GB300 (sm_103a) stencil library.
 *
 * The library evaluates two FP64 3D stencil loop bodies, each in two forms:
 *
 *   as-written ("plain")  the loop body exactly as a directive-style code states it: one
 *                         thread per point, every statement evaluated on its own with its
 *                         own loads and its own recomputation of shared subexpressions;
 *   saturated             the same values after the rewrites of equality saturation
 *                         (paper Sec. V-A, Table I: FMA formation, commutativity,
 *                         associativity, constant folding; Sec. IV-B: extraction with
 *                         common subexpressions counted once) and "bulk load"
 *                         (Sec. VI-B: every load moved to the earliest point, ahead of the
 *                         arithmetic), here extended across neighbouring iterations.
 *
 * Both forms compute the as-written value up to floating-point rounding; equality
 * saturation preserves semantics (Sec. IV). The two loop bodies are:
 *
 *  (1) RHS of the 3D compressible Euler equations with 4th-order artificial dissipation,
 *      the halo-CFD kernel shape of NPB BT/LU/SP (Table II). Conserved variables
 *      U = (rho, m_x, m_y, m_z, E), ideal gas with ratio gamma. At each interior point p
 *      and component c:
 *        R_c(p) = - sum_d (F_{d,c}(p+e_d) - F_{d,c}(p-e_d)) / (2 h_d)
 *                 - eps * sum_d (U_c(p-2e_d) - 4U_c(p-e_d) + 6U_c(p) - 4U_c(p+e_d) + U_c(p+2e_d))
 *      with v_d = m_d/rho, P = (gamma-1)(E - |m|^2/(2 rho)) and
 *        F_d = [m_d, m_x v_d + P[d=x], m_y v_d + P[d=y], m_z v_d + P[d=z], (E+P) v_d].
 *  (2) Variable-coefficient 25-point (radius 4) star stencil, the halo-Jacobi shape of
 *      SPEC ACCEL ostencil (Table III):
 *        out(p) = sum_d sum_{o=1..4} c[d][o-1] * a(p) * (u(p+o e_d) - 2u(p) + u(p-o e_d)).
 *
 * Conventions common to every entry point
 *  - All arrays are FP64 in device memory owned by the caller. The library never
 *    allocates device memory on these paths and keeps no pointer after a call returns.
 *  - x is the unit-stride axis. Inputs are halo-extended arrays addressed from their
 *    corner cell: element (i, j, k) of component c of an input is at
 *        base[c*in_sc + k*in_sz + j*in_sy + i],   0 <= i < nx+2*halo, ...
 *    and interior point (i, j, k) is extended element (i+halo, j+halo, k+halo).
 *    Outputs are addressed from interior point (0, 0, 0):
 *        out[c*out_sc + k*out_sz + j*out_sy + i],  0 <= i < nx, ...
 *    Only interior points are written; nothing else in the output buffer is touched.
 *  - Calls are asynchronous on `stream` (NULL = the legacy default stream). Argument
 *    checks run on the host before any launch; a failed check launches nothing and
 *    returns a status. Launch failures return ACS_ERR_CUDA. `acs_last_error()` gives a
 *    human-readable reason for the last failure of the calling thread.
 *  - Inputs and outputs must not overlap in memory (ACS_ERR_ALIAS).
 *  - The saturated RHS computes 1/rho with a refined hardware reciprocal estimate for
 *    normal |rho| in [2^-1000, 2^1001), faithful (within 1 ulp of the correctly rounded 1/rho),
 *    and falls back to an IEEE division otherwise.
 */
#ifndef ACS_H
#define ACS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream handle; this is the type behind cudaStream_t. */
typedef struct CUstream_st *acs_stream;

typedef enum acs_status {
    ACS_OK = 0,
    ACS_ERR_INVALID = 1,     /* null pointer, bad size, stride or parameter */
    ACS_ERR_ALIGN = 2,       /* a pointer or stride breaks an alignment the kernel needs */
    ACS_ERR_CUDA = 3,        /* a CUDA runtime call or a kernel launch failed */
    ACS_ERR_UNSUPPORTED = 4, /* valid request that the library does not implement */
    ACS_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    ACS_ERR_NOMODEL = 6,     /* no ranker model was supplied where one is required */
    ACS_ERR_ALIAS = 7,       /* an output overlaps an input */
    ACS_ERR_WORKSPACE = 8    /* workspace missing or too small */
} acs_status;

/* Geometry of one grid (see the addressing rules above). */
typedef struct acs_grid {
    int nx, ny, nz;                    /* interior points per axis, each >= 1 */
    int halo;                          /* ghost layers of the inputs on every side */
    long long in_sy, in_sz, in_sc;     /* input element strides: row, plane, component */
    long long out_sy, out_sz, out_sc;  /* output element strides: row, plane, component */
} acs_grid;

/* Physical parameters of the RHS: ratio of specific heats, dissipation weight, spacing. */
typedef struct acs_rhs_params {
    double gamma;
    double eps;
    double h[3];                       /* grid spacing along x, y, z; each nonzero */
} acs_rhs_params;

/*
 * Code versions of the RHS loop body (paper Sec. VII, the four variants compared there,
 * plus the two ends of the ladder):
 *   ACS_FORM_AS_WRITTEN  the original body (acs_rhs_plain)
 *   ACS_FORM_CSE         shared subexpressions counted once (Sec. IV-B), temporaries at
 *                        first use (Sec. VI-A), no rewriting rules
 *   ACS_FORM_CSE_SAT     CSE plus the Table I rules (FMA, ASSOC/COMM, constant folding)
 *   ACS_FORM_CSE_BULK    CSE plus bulk load (Sec. VI-B): all 65 loads before the first store
 *   ACS_FORM_ACCSAT      CSE + SAT + BULK (the paper's full tool)
 *   ACS_FORM_SATURATED   the cross-iteration saturated kernel (acs_rhs_saturated)
 * The four middle forms rewrite each iteration on its own, one thread per point.
 */
typedef enum acs_form {
    ACS_FORM_AS_WRITTEN = 0,
    ACS_FORM_CSE = 1,
    ACS_FORM_CSE_SAT = 2,
    ACS_FORM_CSE_BULK = 3,
    ACS_FORM_ACCSAT = 4,
    ACS_FORM_SATURATED = 5
} acs_form;

/* A compiled rewriter variant (acs_variant_build); opaque. */
typedef struct acs_variant_module *acs_variant_handle;

/* Launch shape of a saturated kernel. A NULL tile selects the built-in default (or the shape
 * the autotuner recorded for the grid size). */
typedef struct acs_tile {
    int bx;       /* threads (points) along x per block: 16, 32 or 64 */
    int by;       /* threads (points) along y per block: 4, 8 or 16 */
    int kchunk;   /* z-planes marched by one block; 0 = pick from the grid size */
    int flags;    /* 0, ACS_TILE_BALANCED and / or ACS_TILE_TMA (single-grid saturated calls) */
} acs_tile;

/* acs_tile.flags: instead of one block per (column tile, z-chunk), launch one block per
 * resident slot of the device and give every block an equal contiguous share of the
 * (column tile, z-plane) work, so that no wave is partly filled; kchunk is then ignored.
 * Accepted by acs_rhs_saturated, acs_rhs_saturated_host, acs_stencil_saturated and the
 * single-grid autotuners; the batch entry points reject it (their blocks already take work
 * from a queue). */
#define ACS_TILE_BALANCED 1
/* acs_tile.flags: stage each xy-plane of the input into shared memory with one tensor copy
 * (TMA, cp.async.bulk.tensor) completing on an mbarrier, instead of element-wise cp.async.
 * Accepted by the single-grid saturated calls, their autotuners and star-stencil batches
 * (acs_batch_prepare, acs_autotune_batch: per grid; RHS batches and acs_batch_run_static reject
 * it). Used where the layout allows it (16-byte aligned input, row, plane and component strides
 * that are multiples of 2 elements, even halo); other layouts, or other grids of a batch, are
 * staged element-wise, with the same results. Waits on the mbarriers are bounded (about one
 * second); one that runs out is counted (acs_wait_timeouts) and the call's results are then
 * wrong, but the kernel ends. */
#define ACS_TILE_TMA 2

/*
 * acs_rhs_plain - as-written RHS, loop body (1) evaluated statement by statement.
 *   U      input, 5 components, halo >= 2        (read only)
 *   R      output, 5 components, interior only   (written)
 *   g      geometry; in_sc and out_sc separate the 5 components
 *   p      gamma, eps, h
 * Alignment: 8-byte aligned pointers. Returns ACS_OK or an error status.
 */
acs_status acs_rhs_plain(const double *U, double *R, const acs_grid *g, const acs_rhs_params *p,
                         acs_stream stream);

/*
 * acs_rhs_saturated - the saturated RHS: per-point fluxes computed once and shared with
 * the six neighbours, one reciprocal per point, dissipation reassociated as
 * sum(U at +-2) - 4 sum(U at +-1) + 18 U, FMA throughout, and every plane of U staged in
 * shared memory ahead of the arithmetic (bulk load). With equal spacing on the three axes
 * (h within 2^-65 .. 2^63) the library's kernel folds -1/(2h) into the fluxes where they are
 * formed (114 FP64 operations per point instead of 116); both forms equal the as-written
 * definition over the reals and differ from it only by rounding. Same arguments as
 * acs_rhs_plain plus
 *   tile     launch shape or NULL (the autotuned shape for this grid size if acs_autotune_rhs
 *            recorded one, else 16 x 16 with the balanced schedule and TMA plane staging where
 *            the layout allows it).
 *   variant  NULL for the library's own saturated kernel, or a march-scope rewriter variant
 *            (acs_variant_generate with ACS_SCOPE_MARCH, acs_variant_build), for instance the
 *            one the learned ranker put first (acs_variant_rank). A variant is compiled for its
 *            block shape, staging and schedule: `tile` must then be NULL or carry the
 *            variant's bx, by and flags (only kchunk is free, for the z-chunk schedule).
 *            ACS_ERR_INVALID for an iteration-scope variant or a mismatched tile;
 *            ACS_ERR_UNSUPPORTED for a TMA-staged variant on a layout TMA cannot copy.
 */
acs_status acs_rhs_saturated(const double *U, double *R, const acs_grid *g, const acs_rhs_params *p,
                             const acs_tile *tile, acs_variant_handle variant, acs_stream stream);

/*
 * acs_rhs_saturated_host - the saturated RHS on HOST arrays, streamed through the GPU in
 * z-slabs of `slab` planes (0 = 12) so that uploads, kernels and downloads overlap.
 *   U, R   host arrays in compact layout (in_sy = nx + 2 halo, in_sz = in_sy (ny + 2 halo),
 *          out_sy = nx, out_sz = nx ny; component strides free). Page-locked memory is
 *          needed for the copies to overlap; pageable memory works but serialises.
 *   tile   launch shape of the slab kernels or NULL (16 x 16, balanced schedule, TMA staging).
 *   ws     device workspace of acs_rhs_host_workspace_bytes(g, slab) bytes (three input and
 *          three output slab buffers), 16-byte aligned.
 * Uploads, halo-plane copies, the slab kernels (alternating between two streams) and downloads
 * run on five library-owned streams per device, ordered by events (concurrent calls on one
 * device share those streams, so their copies queue behind each other). The first upload
 * waits for the work already enqueued on `stream`, and on return `stream` is ordered after the
 * last download (so a later cudaStreamSynchronize(stream) means R is complete on the host). Each input plane
 * crosses the host link once (the halo planes shared by consecutive slabs are copied on the
 * device by a small kernel). The upload of a slab waits for the download of the slab three
 * before it, so uploads run at most three slabs ahead of downloads.
 */
size_t acs_rhs_host_workspace_bytes(const acs_grid *g, int slab);
acs_status acs_rhs_saturated_host(const double *U, double *R, const acs_grid *g, const acs_rhs_params *p,
                                  const acs_tile *tile, int slab, void *ws, size_t ws_bytes, acs_stream stream);

/*
 * acs_rhs_form - the RHS in one of the acs_form code versions (same arguments as
 * acs_rhs_saturated; `tile` is used by ACS_FORM_SATURATED only). ACS_ERR_INVALID for an
 * unknown form.
 */
acs_status acs_rhs_form(const double *U, double *R, const acs_grid *g, const acs_rhs_params *p, int form,
                        const acs_tile *tile, acs_stream stream);

/*
 * acs_stencil_plain - as-written 25-point star stencil, loop body (2).
 *   u, a   inputs with the same geometry, halo >= 4 (only a at interior points is read)
 *   out    output, interior only
 *   c      12 host doubles, c[4*d + (o-1)] for axis d = 0..2 (x, y, z), offset o = 1..4
 */
acs_status acs_stencil_plain(const double *u, const double *a, double *out, const acs_grid *g,
                             const double *c, acs_stream stream);

/*
 * acs_stencil_saturated - the saturated star stencil:
 *   out = a(p) * (C0 u(p) + sum_d sum_o c[d][o] (u(p+o e_d) + u(p-o e_d))),
 *   C0 = -2 sum c (folded on the host), FMA throughout, u planes staged in shared memory
 *   and reused by the 9 z-offsets as the block marches along z.
 *   tile   launch shape or NULL (the autotuned shape for this grid size if
 *          acs_autotune_stencil recorded one, else 32 x 8, z-chunks from the grid size, TMA
 *          plane staging where the layout allows it).
 */
acs_status acs_stencil_saturated(const double *u, const double *a, double *out, const acs_grid *g,
                                 const double *c, const acs_tile *tile, acs_stream stream);

/* ---------------------------------------------------------------------------------------
 * Batched persistent launch (many grids of uneven sizes, one kernel launch).
 *
 * Each grid is cut into work units (tile x z-chunk); a persistent grid of blocks pops units
 * from an atomic counter kept in a caller-provided device workspace, so any number of
 * grids costs one launch. Grids run largest first; the smallest ones, whose units make up
 * about the last two waves of blocks, use z-chunks a quarter of tile->kchunk long. Use: acs_batch_workspace_bytes(n) -> allocate -> acs_batch_prepare
 * (validates every item, uploads the unit table, synchronises `stream`) -> acs_batch_launch
 * as often as needed. acs_batch_launch enqueues a memset of the counter and one kernel on
 * `stream`; it may be captured in a CUDA graph. The items' buffers and the workspace must
 * stay valid while launches are in flight; launches sharing one workspace must not overlap.
 * ------------------------------------------------------------------------------------- */
typedef enum acs_kind {
    ACS_KIND_RHS = 0,      /* loop body (1); params: const acs_rhs_params*  */
    ACS_KIND_STENCIL = 1   /* loop body (2); params: const double[12] weights */
} acs_kind;

typedef struct acs_batch_item {
    const double *in0;     /* U (RHS) or u (stencil), device */
    const double *in1;     /* NULL (RHS) or a (stencil), device */
    double *out;           /* R (RHS) or out (stencil), device */
    acs_grid g;            /* this grid's geometry (addressing rules above) */
} acs_batch_item;

typedef struct acs_batch_plan {      /* filled by acs_batch_prepare; treat as opaque */
    int kind;
    int n;
    acs_tile tile;
    long long total_units;
    void *ws;
    size_t ws_bytes;
} acs_batch_plan;

/* Device workspace bytes acs_batch_prepare needs for n grids (0 if n < 1). */
size_t acs_batch_workspace_bytes(int n);

/*
 * acs_batch_prepare - check n >= 1 items of one kind (each as its single-grid entry point
 * would, including the alias check), order them largest first, and upload the unit table
 * into `ws` (16-byte aligned device memory of at least acs_batch_workspace_bytes(n) bytes:
 * ACS_ERR_ALIGN / ACS_ERR_WORKSPACE otherwise). `tile` NULL = 32 x 8 with z-chunks of 16
 * planes; tile->flags may be ACS_TILE_TMA for a star-stencil batch, which encodes a tensor map
 * per grid into the workspace (grids of even row and plane pitch are then staged by tensor
 * copies, the others element-wise). On success fills `plan`.
 */
acs_status acs_batch_prepare(const acs_batch_item *items, int n, int kind, const acs_tile *tile, void *ws,
                             size_t ws_bytes, acs_batch_plan *plan, acs_stream stream);

/* acs_batch_launch - run a prepared batch; `params` as given for its kind above. */
acs_status acs_batch_launch(const acs_batch_plan *plan, const void *params, acs_stream stream);

/*
 * acs_batch_run_static - a batch (as acs_batch_prepare + acs_batch_launch) that allocates
 * nothing and takes no workspace. The paper has no counterpart; it serves callers that
 * cannot call cudaMalloc when they run a batch: applications that give this library a fixed
 * device budget through their own allocator, or time-critical loops that cannot accept the
 * synchronisation an allocation may cause. The scratch (work counter and unit table) lives
 * in a fixed device array inside the library, sized for ACS_BATCH_STATIC_MAX grids, held on
 * every GPU that loads the library until the process exits. n > ACS_BATCH_STATIC_MAX
 * returns ACS_ERR_WORKSPACE without launching. The first call on a device looks up the
 * array's device address with that device current. Every call uploads the unit table with a
 * host copy and synchronises `stream` (as acs_batch_prepare does), then zeroes the counter and
 * launches, so no call can be made while `stream` is being captured into a CUDA graph: callers
 * that want a graph use acs_batch_prepare + acs_batch_launch. Calls from several host threads
 * are serialised from upload to launch by a library mutex; calls share the array, so calls
 * whose kernels overlap on the GPU (streams not ordered against each other) race.
 * `tile` NULL = 32 x 8, z-chunks of 16; `params` as for the kind.
 */
#define ACS_BATCH_STATIC_MAX 256
acs_status acs_batch_run_static(const acs_batch_item *items, int n, int kind, const acs_tile *tile,
                                const void *params, acs_stream stream);

/* ---------------------------------------------------------------------------------------
 * Launch-shape autotuner. Each call times every built tile with several z-chunk lengths (and,
 * for the single-grid tuners, the balanced schedule, ACS_TILE_BALANCED) on the caller's buffers (outputs are overwritten, `stream` is synchronised: do not capture),
 * returns the fastest shape in `best` (and its time in `best_ms` if non-NULL) and records it
 * in a process-wide cache keyed by the workload shape. acs_rhs_saturated and
 * acs_stencil_saturated called with tile == NULL use the cached shape for their grid size.
 * ------------------------------------------------------------------------------------- */
acs_status acs_autotune_rhs(const double *U, double *R, const acs_grid *g, const acs_rhs_params *p,
                            acs_tile *best, float *best_ms, acs_stream stream);
acs_status acs_autotune_stencil(const double *u, const double *a, double *out, const acs_grid *g,
                                const double *c, acs_tile *best, float *best_ms, acs_stream stream);
acs_status acs_autotune_batch(const acs_batch_item *items, int n, int kind, const void *params, void *ws,
                              size_t ws_bytes, acs_tile *best, float *best_ms, acs_stream stream);
/* Save / load (merge) / clear the tuning cache; a small versioned text file ("acs-tune-cache 2"
 * lines: bx by kchunk flags ms key; version-1 files, without the flags column, still load). */
acs_status acs_tune_cache_save(const char *path);
acs_status acs_tune_cache_load(const char *path);
void acs_tune_cache_clear(void);
int acs_tune_cache_size(void);

/* ---------------------------------------------------------------------------------------
 * Host rewriter of the RHS body (paper Sec. IV-VI) and its learned ranker.
 *
 * acs_variant_generate builds a body in an e-graph, saturates it with the Table I rules plus
 * the rule families the paper leaves off (division, distributivity, subtraction/negation) and,
 * in the march scope, like-term collection, drawing the families, their order and the limits
 * (at most 10,000 e-nodes, 10 iterations) from (seed, index), extracts one program under the
 * paper's cost model (Sec. V-B) with per-variant cost factors, and emits it as a CUDA kernel.
 * Two scopes:
 *   ACS_SCOPE_ITERATION  the paper's scope (Sec. IV-A): the as-written loop body of one point,
 *                        rewritten on its own, one thread per point (first-use or bulk-load
 *                        order, Sec. VI); index 0 is the body with only hash-consing (CSE).
 *   ACS_SCOPE_MARCH      across neighbouring iterations: the body split at the flux of a point
 *                        (the subexpression every statement differencing that point shares)
 *                        into a flux program, evaluated once per point, and a combine program
 *                        per component, each saturated and extracted on its own e-graph and
 *                        emitted into the saturated march kernel (x/y fluxes shared through
 *                        shared memory, z fluxes through registers, planes staged ahead). A
 *                        variant also draws its instruction lowering, tile, plane staging and
 *                        schedule (info->block_x, block_y, flags). index 0: hash-consing only,
 *                        16 x 16, balanced, TMA.
 * Host only; no GPU is touched. `src` / `dag` may be NULL; a too-small buffer returns
 * ACS_ERR_INVALID with the needed size in info->src_bytes / dag_bytes.
 * The DAG text has one line "id op a b c payload" per extracted node in emission order
 * (op in const, param, load, add, sub, mul, div, fma, neg, rcp, flux; fma(a,b,c) = a*b + c;
 * const payload = IEEE bits; load payload = component * 13 + point, points 0 = p,
 * 1..6 = +x,-x,+y,-y,+z,-z, 7..12 = the same at distance 2; param 0 gamma, 1 eps,
 * 2..4 = 1/(2h)) and a line "R c id" per output component. In the march scope the text has
 * two sections: "flux" (loads of point 0 only) ending with lines "F d s id" (F_d,s, d = 0..2
 * for x, y, z, s = 1..4), then "combine", whose flux nodes are the neighbour fluxes (payload
 * d * 8 + (s - 1) * 2 + side, side 0 = p + e_d, 1 = p - e_d), ending with the "R c id" lines.
 * ------------------------------------------------------------------------------------- */
#define ACS_VARIANT_NFEAT 20
typedef enum acs_scope {
    ACS_SCOPE_ITERATION = 0,
    ACS_SCOPE_MARCH = 1
} acs_scope;
/* Static features (names from acs_variant_feature_name), per interior point:
 *  0 paper_cost  1 n_add (add + sub)  2 n_mul  3 n_fma  4 n_div (IEEE divisions and reciprocals)
 *  5 n_neg  6 n_load (march: combine reads + 5)  7 n_load_x (march: combine loads)
 *  8 n_load_yz (march: neighbour-flux reads)  9 n_nodes  10 max_live  11 bulk  12 pipe
 *  13 block_x  14 regs (filled by the caller after acs_variant_build)  15 dp_ops_est
 *  16 block_y  17 tma  18 balanced  19 n_rcp_fast (refined reciprocals).
 * March counts exclude operations on constants and parameters only (hoisted by the compiler). */
typedef struct acs_variant_info {
    float feats[ACS_VARIANT_NFEAT];
    double cost;                     /* the paper's cost of the extracted DAG(s), shared nodes once */
    int enodes, eclasses, iterations;
    int scope;                       /* acs_scope */
    int block_x, block_y;            /* block shape (iteration scope: block_x x 256/block_x threads) */
    int flags;                       /* march scope: ACS_TILE_BALANCED / ACS_TILE_TMA it is built for */
    long long src_bytes, dag_bytes;  /* buffer sizes needed (including the terminating 0) */
} acs_variant_info;

acs_status acs_variant_generate(unsigned long long seed, int index, int scope, char *src, size_t src_len, char *dag,
                                size_t dag_len, acs_variant_info *info);
const char *acs_variant_feature_name(int i);

/* Compile a generated variant (src and the info acs_variant_generate filled) with NVRTC for
 * sm_103a (FMA contraction off, so the extracted operations are what runs) and load it on the
 * current device; `regs` receives the register count. With out == NULL the source is only
 * compiled (no device is needed), to check it. ACS_ERR_UNSUPPORTED if libnvrtc cannot be
 * loaded, ACS_ERR_INVALID with the compiler's log in acs_last_error() if compilation fails. */
acs_status acs_variant_build(const char *src, const acs_variant_info *info, acs_variant_handle *out, int *regs);
/* Run a loaded variant on a grid (same geometry rules as acs_rhs_plain); a march-scope variant
 * runs with its own tile and flags (as acs_rhs_saturated with tile NULL). */
acs_status acs_variant_launch(acs_variant_handle h, const double *U, double *R, const acs_grid *g,
                              const acs_rhs_params *p, acs_stream stream);
/* Unload a variant; call it only after every launch of the variant has completed. */
void acs_variant_free(acs_variant_handle h);

/* FP32 MLP ranker (3 layers, ReLU, hidden width `hidden`): parameters and workspace sizes. */
size_t acs_ranker_param_count(int n_feats, int hidden);
size_t acs_ranker_workspace_bytes(int n, int n_feats, int hidden);
/* Train on n variants: feats (device, n x n_feats floats), times_ms (device, n floats > 0);
 * writes the model into params (device, acs_ranker_param_count floats). Full-batch Adam on the
 * weighted squared error of the standardised log time t: sample weight exp(-fast_weight t_i)
 * normalised to mean 1 (0 = plain mean squared error; larger values weigh the fast variants,
 * which decide the pick, more; at most 8). Deterministic for a given seed. epochs == 0 writes
 * the initial model only (standardisation statistics and seeded initial weights).
 * Parameter layout (floats): mu[F] sd[F] tmu tsd W1[H][F] b1[H] W2[H][H] b2[H] w3[H] b3. */
acs_status acs_ranker_train(const float *feats, const float *times_ms, int n, int n_feats, int hidden, int epochs,
                            float lr, float fast_weight, unsigned long long seed, float *params, void *ws,
                            size_t ws_bytes, acs_stream stream);
/* Gradient of that training loss (with the statistics stored in params and the same sample
 * weights) with respect to every parameter at `params`, without updating them: grad (device,
 * acs_ranker_param_count floats; 0 for mu, sd, tmu, tsd). Same kernels as one training epoch.
 * ws as for acs_ranker_train. Synchronises `stream`. */
acs_status acs_ranker_gradient(const float *feats, const float *times_ms, int n, int n_feats, int hidden,
                               const float *params, float fast_weight, float *grad, void *ws, size_t ws_bytes,
                               acs_stream stream);
typedef struct acs_ranker_model {
    int n_feats;
    int hidden;
    const float *params;   /* device */
} acs_ranker_model;
/* Rank n variants, fastest first. feats: device (n x n_feats); scores_dev: device scratch of
 * n floats; order_out / score_out: host arrays of n (score = predicted ms, or the analytical
 * cost feats[i][0] when model is NULL). Synchronises `stream`. */
acs_status acs_variant_rank(const float *feats, int n, int n_feats, const acs_ranker_model *model, float *scores_dev,
                            int *order_out, float *score_out, acs_stream stream);
/* Save a trained model to a small versioned text file ("acs-ranker-model 1", then "F H P",
 * then the P parameters in hexadecimal floating point, so a load restores the same bits), and
 * load one back into device memory: params (device) of `capacity` floats, or NULL to read
 * only n_feats / hidden (either may be NULL). ACS_ERR_INVALID for an unreadable or malformed
 * file, ACS_ERR_WORKSPACE if the buffer is too small. Synchronous: both first wait for all work
 * on the current device (the model may be written or read on any stream). */
acs_status acs_ranker_save(const char *path, const acs_ranker_model *model);
acs_status acs_ranker_load(const char *path, float *params, size_t capacity, int *n_feats, int *hidden);

/*
 * acs_block_form - the block-assembly body (a third loop body, the many-statement shape of
 * the paper's Listing 2): per interior point 75 outputs from 5 x 5 blocks A, B on the planes
 * k-1, k, k+1 and a scalar G, with t1 = dt q1, t2 = dt q2 and q = 5m + n:
 *   out[q]      = -t2 A_q(k-1) - t1 B_q(k-1) - t1 q3 G [m = n]
 *   out[25 + q] = 2 t1 B_q(k) - q4 t2 A_q(k) + [m = n] (1 + 2 t1 q3 G)
 *   out[50 + q] = t2 A_q(k+1) - t1 B_q(k+1) - t1 q3 G [m = n]
 *   A, B   25 components each (stride g->in_sc), halo >= 1; G one component with the same
 *          row/plane strides; out 75 components (stride g->out_sc)
 *   prm    5 host doubles {dt, q1, q2, q3, q4}
 *   form   ACS_FORM_AS_WRITTEN, ACS_FORM_CSE, ACS_FORM_CSE_BULK or ACS_FORM_SATURATED
 *          (constants folded, every operation an FMA, loads free to move ahead of stores)
 */
acs_status acs_block_form(const double *A, const double *B, const double *G, double *out, const acs_grid *g,
                          const double *prm, int form, acs_stream stream);

/* Static text for a status code. */
const char *acs_status_string(acs_status s);

/*
 * acs_wait_timeouts - how many bounded device-side waits (TMA plane staging) have run out on
 * the current device since the library was loaded; 0 in normal operation. Synchronous: reads a
 * device counter with cudaMemcpy, so call it after the work has completed (for instance after
 * cudaStreamSynchronize). ACS_ERR_INVALID for a NULL count, ACS_ERR_CUDA if the read fails.
 */
acs_status acs_wait_timeouts(unsigned int *count);

/*
 * acs_wait_selftest - run the bounded-wait path once on the current device: one block of 32
 * threads, each waiting with the saturated kernels' own bounded wait (about one second of
 * SM clock cycles) on an mbarrier phase that nothing completes, so every wait runs out. Writes
 * the number of waits that ran out to *timeouts (32 when the path works) and leaves the
 * acs_wait_timeouts counter alone. No copy is issued, so nothing is left in flight. Enqueued on
 * `stream`, which it synchronises (takes about one second). ACS_ERR_INVALID for a NULL
 * timeouts, ACS_ERR_CUDA if the launch or the read fails.
 */
acs_status acs_wait_selftest(unsigned int *timeouts, acs_stream stream);

/*
 * acs_fp64_rate_probe - measure the FP64 pipe: `blocks` x `threads` threads (threads a multiple
 * of 32, at most 1024) each run 8 independent chains of `iters` dependent FMAs whose three
 * operands are registers (the form every FP64 operation of the saturated kernels takes), and
 * store one double each into sink (device, blocks x threads doubles). *ops receives the FP64
 * operations the launch issues (blocks x threads x iters x 8); the caller times the launch on
 * `stream` (CUDA events) to get the pipe's rate, the denominator of the saturated kernels'
 * roofline. Asynchronous.
 */
acs_status acs_fp64_rate_probe(double *sink, int blocks, int threads, int iters, long long *ops, acs_stream stream);

/*
 * acs_rcp_selftest - apply the saturated RHS's reciprocal to n device doubles: y[i] ~ 1/x[i]
 * (a hardware estimate refined by one third-order Newton-Raphson step for normal |x| in
 * [2^-1000, 2^1001), an IEEE division otherwise). For measuring its error against 1/x.
 * Asynchronous; x and y must not overlap.
 */
acs_status acs_rcp_selftest(const double *x, double *y, long long n, acs_stream stream);

/* Reason for the calling thread's most recent failed call ("" if none). */
const char *acs_last_error(void);

/* ABI version of this library (major * 100 + minor). 200: acs_rhs_saturated takes a variant,
 * acs_variant_generate a scope and acs_variant_build the variant's info, acs_variant_info has
 * 20 features and the scope, block and flags fields; the ranker's gradient, model files, the
 * FP64 rate probe and the reciprocal self-test are added. (1xx: 101 added ACS_TILE_BALANCED,
 * ACS_TILE_TMA and acs_wait_timeouts, 102 acs_wait_selftest.) */
int acs_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ACS_H */
