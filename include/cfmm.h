/*
 * cfmm.h -- C ABI of the GB300 (sm_103a) complex-coordinate FMM.
 *
 * Applies 2D/3D Laplace and Helmholtz single- and double-layer potentials to
 * points whose coordinates are complex (Goodwill, Greengard, Hoskins, Rachh,
 * Wang, "Fast Multipole Method with Complex Coordinates"):
 *
 *   out_i = sum_{j: x_j != x_i} K(x_i, x_j) sigma_j
 *         + sum_{j: x_j != x_i} (n_j . grad_y K)(x_i, x_j) tau_j        (Sec. 2.1, 2.3)
 *
 * with the constant-free kernels of Eqs. lap_2d_pot (log r), helm_2d_pot
 * (H_0^(1)(k r)), lap_3d_pot (1/r) and the 3D Helmholtz sum of Sec. 5.3
 * (e^{ikr}/r), continued analytically in the complex distance
 * r = sqrt((x-y).(x-y)) on the principal branch (Sec. 2.1, Def. 3.1).
 * CFMM_GREEN_SCALE multiplies the result by -1/(2 pi), i/4, 1/(4 pi), 1/(4 pi).
 *
 * Every entry point returns (or sets) a status: 0 = OK, negative = error.
 * No C++ exception crosses the ABI. cfmm_last_status()/cfmm_last_error()
 * report the last failure of the calling thread.
 *
 * Memory conventions
 *   - points / normals: row-major [n][dim] float64, real and imaginary parts
 *     in separate arrays (a torch (n, dim) float64 tensor). Host or device
 *     pointers (detected with cudaPointerGetAttributes). The plan copies them.
 *   - densities / out: interleaved complex128 (re, im). densities has layout
 *     [nrhs][ncomp][n] with ncomp = 1 (SLP or DLP) or 2 (SLP sigma then DLP
 *     tau); out has layout [nrhs][n], in the caller's point order, and is
 *     overwritten. Host or device pointers; host buffers are staged through
 *     device memory inside the call (the copies are part of the call).
 *   - the caller owns all buffers it passes; the plan owns its own.
 *
 * Threading: a plan is bound to one CUDA stream and is not re-entrant.
 * Distinct plans may be used concurrently from different threads/streams.
 */
#ifndef CFMM_H
#define CFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
enum {
    CFMM_OK = 0,
    CFMM_EINVAL = -1,      /* bad dim/kernel/k/eps/n/nrhs/options               */
    CFMM_ENONFINITE = -2,  /* NaN or Inf in points or normals                   */
    CFMM_EGEOM = -3,       /* geometry outside the method's assumptions: Re r^2 */
                           /*   <= 0 for a close pair (cfmm_plan checks pairs   */
                           /*   of points near in Morton order)                */
    CFMM_ENOMEM = -4,      /* device allocation failed                          */
    CFMM_ECUDA = -5,       /* CUDA runtime error                                */
    CFMM_ETIMEOUT = -6,    /* a bounded device wait gave up                     */
    CFMM_EUNSUPPORTED = -7 /* valid request this build does not implement       */
};

/* ---- kernel selection (or-ed) ----------------------------------------- */
enum {
    CFMM_LAPLACE = 0,
    CFMM_HELMHOLTZ = 1,
    CFMM_SLP = 1 << 4,          /* single layer (sigma)                      */
    CFMM_DLP = 1 << 5,          /* double layer (tau, needs normals)         */
    CFMM_GREEN_SCALE = 1 << 6   /* multiply by the Green's function constant */
};

/* ---- precision modes -------------------------------------------------- */
enum {
    CFMM_FP64 = 0,   /* every step in float64 / complex128                    */
    CFMM_MIXED = 1,  /* near field and L2P in complex64 arithmetic with       */
                     /* compensated sums; translations stay float64          */
    CFMM_AUTO = 2    /* MIXED when eps >= 1e-5, else FP64                      */
};

enum { CFMM_TOP_FIT = -1 };

typedef struct cfmm_opts {
    int leaf_size;      /* N_s, max points per leaf (Sec. 6.1); 0 = default 64  */
    int sep;            /* separation k = 1..3 of Sec. 6.2/6.5; 0 = default 1;  */
                        /* < 0 = automatic: the smallest k whose Sec. 6.3       */
                        /* Lipschitz limit, times 2, is at least the plan's     */
                        /* Lipschitz estimate (3 if none)                       */
    int precision;      /* CFMM_FP64 / CFMM_MIXED / CFMM_AUTO                   */
    int top_level;      /* top expansion level l0; 0 = automatic rule; > 0 =    */
                        /* that level; CFMM_TOP_FIT (-1) = the rule's level,    */
                        /* then deeper until the 3D Helmholtz order there is    */
                        /* within this library's limit (63; without it such a  */
                        /* plan fails with CFMM_EUNSUPPORTED)                   */
    void* stream;       /* cudaStream_t the plan runs on; NULL = legacy stream  */
} cfmm_opts;

typedef struct cfmm_plan_s* cfmm_plan_t;

/*
 * cfmm_plan: builds the tree on the real parts of the points (Sec. 6.1),
 * the complexified centres (Eq. complexify_center_average), Lists 1-4
 * (Sec. 6.2) and the expansion order per level (Sec. 6.3), all on the GPU.
 *   dim     2 or 3
 *   kernel  CFMM_LAPLACE or CFMM_HELMHOLTZ, or-ed with CFMM_SLP / CFMM_DLP /
 *           CFMM_GREEN_SCALE (default CFMM_SLP)
 *   k       wavenumber kappa > 0 for Helmholtz (ignored for Laplace)
 *   eps     requested relative accuracy, 1e-15 <= eps <= 0.1
 *   pts_re, pts_im  [n][dim] float64 (host or device)
 *   n       number of points (sources = targets), 1 <= n < 2^31
 * Returns NULL on failure (see cfmm_last_status / cfmm_last_error).
 */
cfmm_plan_t cfmm_plan(int dim, int kernel, double k, double eps,
                      const double* pts_re, const double* pts_im, int64_t n);

/*
 * cfmm_plan_ex: as cfmm_plan, with DLP normals ([n][dim] float64 real and
 * imaginary parts; NULL when kernel has no CFMM_DLP) and options (NULL =
 * defaults). The normals are used as given (not renormalised): their length
 * carries the caller's quadrature weight.
 */
cfmm_plan_t cfmm_plan_ex(int dim, int kernel, double k, double eps,
                         const double* pts_re, const double* pts_im,
                         const double* nrm_re, const double* nrm_im,
                         int64_t n, const cfmm_opts* opts);

/*
 * cfmm_plan_targets: a plan that evaluates the potential of m sources at n
 * separate targets (Sec. 2.3 Eq. evaluation_problem with distinct x_i and
 * y_j; the targets may carry their own imaginary parts, the "two different
 * functions psi" of the remark after Lemma 4.1.1, and the Lipschitz condition
 * then holds for both). The tree, centres, lists and orders are built on the
 * m + n points together (sources first); the targets enter the expansions
 * with zero density, and a source that coincides with a target is skipped
 * for it, as in the direct sum.
 *   src_re/src_im [m][dim], nrm_re/nrm_im [m][dim] (source normals; NULL
 *   without CFMM_DLP), trg_re/trg_im [n][dim], float64, host or device.
 * cfmm_apply on such a plan takes densities [nrhs][ncomp][m] and writes out
 * [nrhs][n] (the targets, in the caller's order). Returns NULL on failure.
 */
cfmm_plan_t cfmm_plan_targets(int dim, int kernel, double k, double eps,
                              const double* src_re, const double* src_im,
                              const double* nrm_re, const double* nrm_im, int64_t m,
                              const double* trg_re, const double* trg_im, int64_t n,
                              const cfmm_opts* opts);

/*
 * cfmm_apply: one FMM pass (the eight steps of Sec. 6.4) for nrhs
 * right-hand sides. densities: [nrhs][ncomp][n] complex128; out: [nrhs][n]
 * complex128 (overwritten). Host or device pointers. Asynchronous on the
 * plan's stream for device buffers; returns after the result is in `out`
 * for host buffers. Returns 0 or a negative status.
 */
int cfmm_apply(cfmm_plan_t plan, const double* densities, int nrhs, double* out);

/*
 * cfmm_apply_grad: as cfmm_apply, and also the target gradient of the result,
 *   grad_i = grad_x [ sum_j K(x, y_j) sigma_j + (n_j . grad_y K)(x, y_j) tau_j ] at x = x_i,
 * whose components along a target normal give the normal derivatives S' and
 * D' of Sec. 2.1 (off the surface; on it, the discrete sums of the same
 * kernels). The expansions are those of cfmm_apply; the evaluation steps are
 * differentiated: the near field pair by pair (grad_x K = (K'/r) d, grad_x
 * (n . grad_y K) = -(K'/r) n - ((K'' - K'/r)/r^2)(n.d) d with d = x - y), M2P
 * and L2P through the derivative relations of their expansion functions.
 * The gradient is computed in FP64 (also on a MIXED plan, whose potential
 * keeps its mixed-precision near field and L2P).
 *   out  [nrhs][n_out] complex128 potential, or NULL;
 *   grad [nrhs][dim][n_out] complex128, d/dx_1, .., d/dx_dim at the targets.
 * n_out = n (targets are the sources) or the plan's separate target count.
 * Host or device pointers, as cfmm_apply. Returns 0 or a negative status.
 */
int cfmm_apply_grad(cfmm_plan_t plan, const double* densities, int nrhs, double* out, double* grad);

/*
 * cfmm_apply_capture: records one cfmm_apply/*
 * cfmm_apply_capture: records one cfmm_apply of device buffers (densities,
 * out: device pointers, which must stay valid while the graph is used) into a
 * CUDA graph owned by the plan, replacing any earlier one. The plan must have
 * been created with a non-NULL stream. Nothing runs during capture.
 * cfmm_apply_replay: launches the captured graph on the plan's stream
 * (asynchronous); the result overwrites the captured `out`.
 * Both return 0 or a negative status.
 */
int cfmm_apply_capture(cfmm_plan_t plan, const double* densities, int nrhs, double* out);
int cfmm_apply_replay(cfmm_plan_t plan);

/*
 * Batches of geometries. The paper applies one geometry at a time; a batched
 * solve applies many resident plans (uneven sizes) per step, and one CUDA
 * graph over all of them lets the small geometries' kernels overlap.
 *
 * cfmm_batch_capture: applies each of the `count` plans once eagerly (device
 * buffers densities[i] [nrhs[i]][ncomp_i][n_i] and out[i] [nrhs[i]][n_i]
 * complex128, as in cfmm_apply; `out` holds that result on return), then
 * records the same applies into ONE CUDA graph: `stream` (non-NULL) forks to
 * each plan's stream, the plan's apply runs there, and `stream` joins them.
 * Plans on different streams become concurrent branches; plans sharing a
 * stream run in array order. Every plan needs a non-NULL stream and must live
 * on the current device. The graph keeps the pointers: until
 * cfmm_batch_destroy, the buffers must stay valid, and no member plan may be
 * destroyed or applied with a larger nrhs than captured (that regrows its
 * workspaces). Returns NULL on failure (see cfmm_last_status).
 * cfmm_batch_replay: launches the graph on `stream` (asynchronous); each
 * out[i] is overwritten with the apply of what densities[i] then holds.
 * cfmm_batch_kernels: kernel nodes in the graph (kernels per replay).
 * cfmm_batch_destroy: waits for `stream`, frees the graph; NULL is OK.
 */
typedef struct cfmm_batch_s* cfmm_batch_t;
cfmm_batch_t cfmm_batch_capture(const cfmm_plan_t* plans, int count, const double* const* densities,
                                const int* nrhs, double* const* out, void* stream);
int cfmm_batch_replay(cfmm_batch_t batch);
int64_t cfmm_batch_kernels(cfmm_batch_t batch);
int cfmm_batch_destroy(cfmm_batch_t batch);

/* cfmm_destroy: frees the plan; NULL is OK. */
int cfmm_destroy(cfmm_plan_t plan);

/*
 * cfmm_direct: the direct O(N M) sum of Sec. 2.3 (Eq. evaluation_problem and
 * its double-layer form) on the GPU, skipping pairs with x - y == 0.
 *   src_re/src_im [m][dim], trg_re/trg_im [n][dim], nrm_re/nrm_im [m][dim]
 *   (NULL without CFMM_DLP); densities [nrhs][ncomp][m]; out [nrhs][n].
 *   All device pointers. precision CFMM_FP64 or CFMM_MIXED.
 *   stream: cudaStream_t or NULL. Asynchronous.
 */
int cfmm_direct(int dim, int kernel, double k,
                const double* src_re, const double* src_im,
                const double* nrm_re, const double* nrm_im, int64_t m,
                const double* trg_re, const double* trg_im, int64_t n,
                const double* densities, int nrhs, double* out,
                int precision, void* stream);

/*
 * cfmm_direct_noalloc: the same direct sum as cfmm_direct (FP64), for callers
 * that cannot allocate device memory while they run -- a program that gave
 * its whole device-memory budget to a pool up front, so an allocation by this
 * library would fail, or a latency-critical loop in which cudaMalloc/cudaFree
 * (which may synchronise the device) are not acceptable. The paper has no
 * counterpart: this is a deployment variant of the direct sum.
 *   Arguments, layouts and result as cfmm_direct (device pointers; the caller
 *   passes inputs and output). Allocates nothing: its scratch (SoA copies of
 *   points and normals) is a fixed array of about 4.5 MiB of device memory
 *   inside the library, held by every GPU that loads the library until exit.
 *   Limits: m <= 32768 sources and n <= 32768 targets; larger requests
 *   return CFMM_EINVAL without touching the GPU.
 *   All calls share that array: calls that overlap on the GPU (other
 *   streams, other host threads) race; serialise them. Each call overwrites
 *   what it reads, so nothing needs clearing between calls.
 *   The first call on a device looks up the array's address and uploads the
 *   library's constant tables; make it before any stream capture.
 *   stream: cudaStream_t or NULL. Asynchronous. Returns 0 or a negative status.
 */
int cfmm_direct_noalloc(int dim, int kernel, double k,
                        const double* src_re, const double* src_im,
                        const double* nrm_re, const double* nrm_im, int64_t m,
                        const double* trg_re, const double* trg_im, int64_t n,
                        const double* densities, int nrhs, double* out, void* stream);

/* ---- introspection (tests and tools) --------------------------------- */
typedef struct cfmm_plan_info {
    int dim, kernel, sep, leaf_size, precision;
    int nlevels;        /* levels 0..nlevels-1                                */
    int nboxes;
    int nleaves;
    int l0;             /* top expansion level                               */
    int64_t n;          /* points of the tree (sources + separate targets)   */
    int64_t list_len[4];/* total entries of Lists 1..4                        */
    int64_t p2p_pairs;  /* sum over leaves of n_target * n_source over List 1 */
    int64_t m2l_pairs;  /* List 2 entries at levels >= l0                     */
    double root_lo[3];
    double root_width;
    double lipschitz;   /* estimate of the Lipschitz constant L of Im x     */
                        /* against Re x (Assumptions 4.1/5.1): max over     */
                        /* pairs at most 32 apart in Morton order of        */
                        /* |Im(x_i - x_j)| / |Re(x_i - x_j)|; the plan      */
                        /* fails with CFMM_EGEOM when it reaches 1          */
    int64_t n_src;      /* sources (n_src = n without separate targets)      */
    int64_t n_trg;      /* separate targets (0: the targets are the sources) */
} cfmm_plan_info;

/* cfmm_plan_get_info: fills *info. */
int cfmm_plan_get_info(cfmm_plan_t plan, cfmm_plan_info* info);

/* cfmm_plan_get_orders: P per level into p[0..nlevels-1] (host array); 2D Helmholtz
 * levels above the top expansion level (no expansions there) read 0. */
int cfmm_plan_get_orders(cfmm_plan_t plan, int* p, int nlevels);

/*
 * cfmm_plan_export_tree: copies the tree into caller host arrays (any may be
 * NULL): perm [n] int64 (sorted position -> input index), keys [n] uint64
 * (sorted Morton keys), box_level/box_start/box_end/box_leaf/box_parent
 * [nboxes] int32, box_prefix [nboxes] uint64, center_re/center_im
 * [nboxes][dim] float64.
 */
int cfmm_plan_export_tree(cfmm_plan_t plan, int64_t* perm, uint64_t* keys,
                          int32_t* box_level, uint64_t* box_prefix,
                          int32_t* box_start, int32_t* box_end,
                          int32_t* box_leaf, int32_t* box_parent,
                          double* center_re, double* center_im);

/*
 * cfmm_plan_export_list: List `which` (1..4) as CSR into host arrays:
 * offsets [nboxes+1] int64 and entries [list_len[which-1]] int32, each box's
 * entries sorted by box index. Either pointer may be NULL.
 */
int cfmm_plan_export_list(cfmm_plan_t plan, int which, int64_t* offsets, int32_t* entries);

/* cfmm_plan_timings: per-step device time of the last cfmm_apply in ms
 * (t[0..nsteps-1], steps: 0 permute, 1 P2M, 2 M2M, 3 M2L, 4 P2L,
 * 5 L2L, 6 P2P, 7 M2P+L2P, 8 unpermute); returns the number of steps. */
int cfmm_plan_timings(cfmm_plan_t plan, double* t, int nsteps);

/* cfmm_plan_set_timing: 0 = off; 1 = record per-step CUDA events during apply
 * (the near field runs beside the far field on the plan's second stream, so
 * concurrent steps share the SMs); 2 = serialised: the near field runs in line
 * on the plan's stream and every step's time is its kernels' alone (slower
 * apply, same result bit for bit). Returns CFMM_EINVAL for other values. */
int cfmm_plan_set_timing(cfmm_plan_t plan, int on);

/* cfmm_launch_count: number of kernels this library launched so far in the
 * calling process (all threads). */
int64_t cfmm_launch_count(void);

/* cfmm_debug_fail_allocs: failure injection for tests (no counterpart in the
 * paper): the next `count` device allocations of the library (plan buffers,
 * workspaces, plan-construction scratch) fail with CFMM_ENOMEM, whichever
 * call makes them; 0 disarms. Returns 0, or CFMM_EINVAL for count < 0. */
int cfmm_debug_fail_allocs(int count);

int cfmm_last_status(void);
const char* cfmm_last_error(void);
const char* cfmm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CFMM_H */
