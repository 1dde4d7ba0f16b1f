/*
 * tdgrav: in-plane self-gravity of an infinitesimally thin disk on a uniform grid, by the
 * B-spline direct method of Wang, Shiue, Wu & Yen (arXiv 1904.07400), on one GB300.
 *
 * What a solve computes (paper Eqs. eqnSigma, eqnF, eqnw, eqnwB):
 *   C          = B-spline coefficients of sigma at order k (Sec. 2.3: C = sigma for k = 1, 2;
 *                two truncated tridiagonal solves, Eqs. z_system and C_system, for k = 3;
 *                for k = 4, 5, the extension Sec. 2.2 and Sec. 2.3 call straightforward,
 *                the same interpolation condition with the stencils (1, 4, 1)/6 and
 *                (1, 76, 230, 76, 1)/384: truncated banded solves along y, then x)
 *   F^x_ij     = G * sum_{i'j'} C_{i'j'} w^x(i - i', j - j')
 *   F^y_ij     = G * sum_{i'j'} C_{i'j'} w^y(i - i', j - j')
 *   w^x(m, n)  = PV int int u (u^2+v^2)^(-3/2) b_k(u/dx + m) b_k(v/dy + n) du dv
 * with b_k the centred cardinal B-spline of order k on the cell (Sec. 2.3: every spline is
 * centred on its cell centre).  The convolution is evaluated exactly (up to rounding) by
 * FFTs on a zero-padded grid (Sec. 4.1: one forward transform of C, two inverse transforms),
 * so no boundary values are needed for an isolated disk.
 *
 * Conventions shared by every entry point:
 *   - Arrays are C-contiguous with shape (nx, ny): element [i * ny + j] is cell (x_i, y_j),
 *     axis 0 is x.  sigma, F^x, F^y, and the adjoint buffers use this layout.
 *   - Element type follows the plan's precision: double for TDG_FP64, float for TDG_FP32
 *     and TDG_FP32_TC16.
 *   - Data pointers are DEVICE pointers on the plan's device, owned by the caller, 16-byte
 *     aligned.  The library never frees them and keeps no reference after a call returns.
 *   - Plans own their kernel spectra, twiddle tables and (unless set with
 *     tdg_set_workspace) their workspace; tdg_destroy frees them.
 *   - Every call returns a tdg_status; nothing throws across this interface.  Launches are
 *     asynchronous on the given stream and the solve entry points do not synchronise the
 *     host; NaN or Inf in the input propagates and is not checked.
 *   - `stream` is a cudaStream_t (0 = the legacy default stream).
 */
#ifndef TDGRAV_H
#define TDGRAV_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TDG_OK = 0,
    TDG_ERR_INVALID_ARG = 1,   /* bad size, order, spacing, null or misaligned pointer   */
    TDG_ERR_UNSUPPORTED = 2,   /* size beyond the supported transform lengths            */
    TDG_ERR_NOT_BUILT = 3,     /* solve before tdg_build_kernel_tables                   */
    TDG_ERR_OOM = 4,           /* device allocation failed                               */
    TDG_ERR_CUDA = 5,          /* a CUDA runtime call failed                             */
    TDG_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up (batched launch)    */
    TDG_ERR_DEVICE_BOUNDS = 7  /* a device-side index check failed (checked builds)      */
} tdg_status;

typedef enum {
    TDG_FP64 = 0,       /* every step in double                                          */
    TDG_FP32 = 1,       /* float transforms, spectra rounded from the FP64 build         */
    TDG_FP32_TC16 = 2   /* float; the column pass runs its radix-16 DFT stages as split
                           hi/lo tensor-core products (TF32 operands, tcgen05.mma),
                           accumulated in FP32                                           */
} tdg_precision;

typedef struct tdg_plan_s* tdg_plan;
typedef struct tdg_batch_s* tdg_batch;
typedef struct CUstream_st* tdg_stream;

/* Create a plan for an nx x ny grid of cells dx x dy, B-spline order 1..5, constant G.
 * Allocates nothing on the device yet.  Errors: INVALID_ARG for order not in 1..5,
 * nx or ny < 1, dx or dy not finite and > 0, G not finite, out == NULL; UNSUPPORTED for
 * nx or ny > 4096, and for TDG_FP32_TC16 unless both sides are multiples of 16 from 128
 * to 4096 and nx > 1024 (the tensor-core column pass takes columns padded to 2048 or 4096
 * cells); CUDA if `device` cannot be selected. */
tdg_status tdg_init(tdg_plan* out, int nx, int ny, int order, double dx, double dy,
                    double G, tdg_precision prec, int device);

/* Build the kernel tables w^x, w^y for all offsets |m| < nx, |n| < ny in FP64 on the
 * device (Sec. 2.1-2.2), place them on the periodic padded grid and transform them into
 * the two kernel spectra, rounded to the plan's precision.  Done once per plan (Sec. 4.2:
 * the kernel integrals are computed once and reused).  Synchronises `stream` before
 * returning (the FP64 temporaries are freed).  Errors: OOM, CUDA. */
tdg_status tdg_build_kernel_tables(tdg_plan p, tdg_stream stream);

/* The same build from quarter tables the caller kept (from tdg_copy_kernel_tables of an
 * earlier plan with the same nx, ny, order, dx, dy; w^x then w^y, each nx x ny FP64
 * row-major on the host).  The in-simulation reuse of the paper's Sec. 4.2: the tables
 * are computed once, and a restarted run skips their quadrature (about 0.25 s at 4096^2)
 * and only places and transforms them.  A spot check of ten entries against the table code
 * rejects tables of another order, cell shape or grid.  Errors: INVALID_ARG (NULL
 * arguments, tables that fail the check), OOM, CUDA. */
tdg_status tdg_build_kernel_tables_from(tdg_plan p, const double* wx, const double* wy, tdg_stream stream);

/* Bytes of device workspace a solve or adjoint of this plan needs. */
size_t tdg_workspace_bytes(const tdg_plan p);

/* Hand the plan a caller-owned workspace of at least tdg_workspace_bytes(p) bytes,
 * 256-byte aligned; the plan then allocates none of its own.  ptr == NULL returns to
 * plan-owned workspace (allocated at the next solve).  Errors: INVALID_ARG. */
tdg_status tdg_set_workspace(tdg_plan p, void* ptr, size_t bytes);

/* The potential in the disk plane, a diagnostic beside the forces (the method itself never
 * forms it, Sec. 1): Phi_ij = -G sum_{i'j'} C_{i'j'} w^phi(i - i', j - j') with
 * w^phi(m, n) = int int b_k(u/dx + m) b_k(v/dy + n) (u^2 + v^2)^(-1/2) du dv (even in m and
 * n), by the same zero-padded convolution with one real spectrum.
 * tdg_build_potential_tables: builds w^phi in FP64 on the device and its spectrum in the
 * plan's precision (hy x P_x values; after tdg_build_kernel_tables, whose twiddles it
 * uses); synchronises `stream`.  Errors: NOT_BUILT, OOM, CUDA.
 * tdg_solve_potential: sigma -> Phi (nx*ny elements each, the plan's type, 16-byte
 * aligned, not aliased), asynchronous on `stream`, in the plan's workspace; every
 * precision form runs the generic kernels.  Errors: INVALID_ARG, NOT_BUILT (no potential
 * spectrum), OOM, CUDA. */
tdg_status tdg_build_potential_tables(tdg_plan p, tdg_stream stream);
tdg_status tdg_solve_potential(tdg_plan p, const void* sigma, void* phi, tdg_stream stream);

/* Diagnostics of Sec. 3 on the device: the radial force F_R = (x F^x + y F^y) / R at the
 * cell centres x_i = x0 + (i + 1/2) dx, y_j = y0 + (j + 1/2) dy (F_R = 0 where R = 0), and
 * the error norms the paper's validation uses (Sec. 3.1), area-weighted:
 * L1 = dx dy sum |e|, L2 = (dx dy sum e^2)^(1/2), Linf = max |e|.
 *   fx, fy   the forces of a solve with this plan (nx*ny elements, the plan's type).
 *   fr       output F_R (nx*ny elements) or NULL.
 *   ref_fx   reference F^x (for instance the analytic force) or NULL; ref_fr the same for F_R.
 *   norms    host array of 6 doubles: L1, L2, Linf of F^x - ref_fx, then of F_R - ref_fr
 *            (zeros when ref_fr is NULL); NULL exactly when ref_fx is NULL.
 * Sums are in FP64 with a fixed reduction order.  With norms, the call synchronises
 * `stream` (the six values are copied to the host); without, it only enqueues.  Errors:
 * INVALID_ARG (NULL or misaligned forces, non-finite origin, neither fr nor norms asked,
 * norms without ref_fx or the reverse, ref_fr without ref_fx), OOM, CUDA. */
tdg_status tdg_radial_diagnostics(tdg_plan p, const void* fx, const void* fy, double x0, double y0, void* fr,
                                  const void* ref_fx, const void* ref_fr, double* norms, tdg_stream stream);

/* sigma -> (F^x, F^y) (Eq. eqnF).  sigma, fx, fy: nx*ny elements each.  fx and fy must
 * not alias sigma or each other.  Errors: INVALID_ARG (null/misaligned), NOT_BUILT, OOM
 * (first call allocates the workspace if none was set), CUDA. */
tdg_status tdg_solve_forces(tdg_plan p, const void* sigma, void* fx, void* fy,
                            tdg_stream stream);

/* `count` independent solves, each with its own plan (any nx, ny, order; FP32 plans on
 * one device), executed by one persistent launch (see tdg_batch_create).  Convenience form:
 * creates a batch, launches it on `stream` and releases it, which synchronises the device
 * before returning.  For repeated solves create the batch once and launch it (that launch
 * is asynchronous).  sigma[d], fx[d], fy[d] follow the layout of tdg_solve_forces for
 * plans[d].  Errors: as tdg_batch_create and tdg_batch_launch. */
tdg_status tdg_solve_forces_batched(const tdg_plan* plans, int count,
                                    const void* const* sigma, void* const* fx,
                                    void* const* fy, tdg_stream stream);

/* A reusable batch of independent solves (meshes or disks of uneven sizes and orders,
 * paper Sec. 1 motivates such uses): per-grid descriptors, one workspace and dependency
 * counters on the device.  The pointers are captured at creation; the plans must outlive
 * the batch and keep their kernel tables.  Errors: INVALID_ARG (NULL or misaligned
 * pointers, mixed devices), NOT_BUILT, UNSUPPORTED (FP64 or TC16 plans, a grid that fits neither
 * persistent kernel), OOM, CUDA. */
tdg_status tdg_batch_create(tdg_batch* out, const tdg_plan* plans, int count,
                            const void* const* sigma, void* const* fx, void* const* fy);

/* Form and knobs of the persistent kernel (picked by the autotuner).  threads 256 or 512:
 * the generic kernel (any grid that fits one block), with radix preference 0 (radix 8
 * first) or 1 (radix 4).  threads 64: the kernel on the transform network's item bodies
 * (every grid FP32 on the network path with sides up to 1024 cells); the second argument
 * is then the number of units per item (1, 2, 4, 8, 16 or 32; a unit is one row, column or
 * inverse row of a 1024-length transform, two of a 512-length one, four of a 256-length
 * one): blocks of 64 threads take the items of each pass in turn, grouped by the pass's
 * line length and in decreasing solve cost within a group, a 1024-length unit on both
 * warps, a 512-length unit one transform per warp, a 256-length unit one per half-warp, the
 * column stashes in tensor memory.
 * Errors: INVALID_ARG, UNSUPPORTED (a grid does not fit; the old setting stays). */
tdg_status tdg_batch_set_config(tdg_batch b, int threads, int radix_pref);

/* Second form of the batch (picked by the autotuner): nstreams > 0 runs each grid's own
 * forward path (the kernels tdg_solve_forces would run for its plan, into the batch's
 * workspace) on `nstreams` internal streams, grids assigned by decreasing cost to the
 * least-loaded stream, forked from and joined back to the launch stream with events (so
 * a launch stays asynchronous and capturable in a CUDA graph).  nstreams = 0 returns to
 * the persistent kernel.  The paper has no counterpart; this exists because grids on the
 * FP32 network path solve faster with their own kernels than inside the persistent
 * generic kernel.  Errors: INVALID_ARG (NULL batch, nstreams outside 0..32), CUDA. */
tdg_status tdg_batch_set_streams(tdg_batch b, int nstreams);

/* One persistent launch solving every grid of the batch on `stream`: a memset of the
 * dependency counters and one kernel, no host synchronisation.  Work items (row groups,
 * frequency columns, inverse-row groups) are taken in pass order; an item waits for its
 * own grid's previous pass with a bounded spin (about one second), after which it sets
 * the batch error word to TDG_ERR_TIMEOUT and is skipped.  Errors: INVALID_ARG, CUDA. */
tdg_status tdg_batch_launch(tdg_batch b, tdg_stream stream);

/* Read and clear the batch's device error word (synchronises).  TDG_OK or TIMEOUT. */
tdg_status tdg_batch_get_error(tdg_batch b);

/* Blocks of the persistent launch, threads per block, total work items and radix
 * preference.  Any out pointer may be NULL. */
tdg_status tdg_batch_info(const tdg_batch b, int* blocks, int* threads, int* items,
                          int* radix_pref);

/* Test hook: completions of grid `grid`'s row pass are not counted by later launches
 * (-1 restores normal operation), so its column items exhaust their bounded wait.
 * Exists to test the timeout path without faulting or hanging the device; applies to
 * the persistent kernel only. */
tdg_status tdg_batch_debug_withhold(tdg_batch b, int grid);

/* Release the batch (synchronises its device). */
tdg_status tdg_batch_destroy(tdg_batch b);

/* Adjoint of tdg_solve_forces: for L = sum(gfx * F^x + gfy * F^y), write
 * gsigma = dL/dsigma = (B-spline solve)^T (correlation of gfx, gfy with the same kernel
 * spectra).  All buffers nx*ny elements.  Errors: as tdg_solve_forces. */
tdg_status tdg_solve_adjoint(tdg_plan p, const void* gfx, const void* gfy, void* gsigma,
                             tdg_stream stream);

/* Read and clear the plan's device error word (synchronises the plan's device).
 * TDG_OK if no device-side check failed since the last call. */
tdg_status tdg_get_device_error(tdg_plan p);

/* Copy the FP64 kernel tables for offsets 0 <= m < nx, 0 <= n < ny (the quadrant that
 * fixes the others by symmetry: w^x odd in m and even in n, w^y even in m and odd in n)
 * into host arrays wx, wy of nx*ny doubles each, row-major [m * ny + n].  Only valid
 * after tdg_build_kernel_tables.  Errors: NOT_BUILT, INVALID_ARG, CUDA. */
tdg_status tdg_copy_kernel_tables(const tdg_plan p, double* wx, double* wy);

/* Evaluate one kernel-table entry w^x(m, n) (component 0), w^y(m, n) (component 1) or the
 * potential kernel w^phi(m, n) (component 2, see tdg_build_potential_tables) on the HOST
 * with the same FP64 code the device build runs.  For tests without a GPU.
 * Errors: INVALID_ARG for bad order/spacing/component or out == NULL. */
tdg_status tdg_kernel_entry_host(int order, int m, int n, double dx, double dy,
                                 int component, double* out);

/* Instrumentation: ask every later forward solve or adjoint of this plan to record the
 * caller-owned CUDA events events[0..count-1] (cudaEvent_t handles) on its stream:
 * events[0] before the first pass and events[i] after pass i (1: row transform, 2: column
 * convolution, 3: row inverse transform), so that the caller can time each kernel on the
 * stream it runs on.  count must be 0 (stop recording; events may be NULL) or 4.  The
 * library never creates, destroys or synchronises these events.  Errors: INVALID_ARG. */
tdg_status tdg_set_pass_events(tdg_plan p, void* const* events, int count);

/* Size of the device array behind tdg_solve_forces_noalloc: 32 MiB. */
#define TDG_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* tdg_solve_forces without any allocation (the paper has no counterpart; this serves
 * callers of the library).  Some callers cannot allocate device memory where they solve:
 * code that runs while another allocator owns the device's free memory, real-time loops
 * that must not hit cudaMalloc's implicit synchronisation, or hosts that forbid device
 * allocations after start-up.  They build plans up front (tdg_init and
 * tdg_build_kernel_tables allocate) and solve here: same inputs, outputs and results as
 * tdg_solve_forces, but the scratch is a fixed device array of TDG_NOALLOC_SCRATCH_BYTES
 * that every GPU loading the library holds until the process exits, and the call makes
 * no cudaMalloc, cudaFree or other allocating call.
 *   - The array's device address is looked up when the plan's kernel tables are built
 *     (tdg_build_kernel_tables, with the plan's device current) and kept in the plan, so
 *     this call itself makes no set-up call.
 *   - All calls share the one array and it keeps the last call's contents.  Calls that
 *     overlap on the GPU (several streams or host threads) race on it: serialise them.
 * Errors: UNSUPPORTED when tdg_workspace_bytes(p) > TDG_NOALLOC_SCRATCH_BYTES (about
 * 1024 x 1024 in FP32, 724 x 724 in FP64); otherwise as tdg_solve_forces. */
tdg_status tdg_solve_forces_noalloc(tdg_plan p, const void* sigma, void* fx, void* fy,
                                    tdg_stream stream);

/* ---------------------------------------------------------------------------------------
 * Slab decomposition of one grid over `world` ranks (Sec. 2.3: the spline solves and the
 * transforms are split over processes in slabs, with transposes between the passes).  For
 * FP32 plans on the transform-network path (tdg_plan_path 2) with nx / 16 >= world.  Every
 * rank builds the same plan on its own device; rank r owns rows [r0, r0 + nrows) of sigma
 * and of the forces, and the two-column tiles [t0, t0 + ntiles) of frequency columns
 * ky = 2 t0 .. (the last rank ends at the Nyquist column).  One solve, on every rank:
 *   1. tdg_slab_rows_forward: sigma rows -> Z row slab;
 *   2. all-to-all of the Z row slab: the chunk for rank q (tdg_slab_partition of q) is
 *      ntiles_q * nrows_r cells at cell offset t0_q * nrows_r; chunks arrive in source order;
 *   3. tdg_slab_unpack_z: the received chunks -> Z column slab;
 *   4. tdg_slab_columns: Z column slab -> G column slab (G_x, then G_y);
 *   5. tdg_slab_pack_g: G column slab -> send buffer, per component one chunk per destination
 *      r of ntiles_self * nrows_r cells, in rank order;
 *   6. all-to-all per component: the chunks received in source order are the G row slab
 *      (component c at cell offset c * tdg_slab_bytes(..., 3) / 32);
 *   7. tdg_slab_rows_inverse: G row slab -> force rows.
 * A cell is 16 bytes (two complex floats).  Buffers are DEVICE pointers on the plan's device,
 * owned by the caller, 16-byte aligned, sized by tdg_slab_bytes; all calls are asynchronous
 * on `stream`.  The result equals tdg_solve_forces on the whole grid.  The paper has no
 * library interface; these calls follow its distribution. */

/* Rows and tiles of `rank` for an nx x ny grid (host only, no device).  Rows come in
 * multiples of 16, the extra ones to the first ranks; tiles likewise.  Any out pointer may
 * be NULL.  Errors: INVALID_ARG (sizes off the network path, world < 1, rank outside
 * 0..world-1, fewer 16-row chunks or tiles than ranks). */
tdg_status tdg_slab_partition(int nx, int ny, int world, int rank, int* r0, int* nrows, int* t0, int* ntiles);

/* Bytes of one of rank's slab buffers: which = 0 Z row slab, 1 Z column slab (the received
 * chunks of step 2 have the same size), 2 G column slab (= the send buffer of step 5),
 * 3 G row slab (both components).  0 for a bad plan, rank or `which`. */
size_t tdg_slab_bytes(const tdg_plan p, int world, int rank, int which);

/* Steps 1, 3, 4, 5 and 7 above.  sigma_rows, fx_rows, fy_rows: nrows x ny floats, row-major
 * (row r0 first).  Errors: INVALID_ARG (NULL or misaligned pointers, fx_rows == fy_rows),
 * NOT_BUILT, UNSUPPORTED (plan off the FP32 network path, bad world or rank), CUDA. */
tdg_status tdg_slab_rows_forward(tdg_plan p, int world, int rank, const void* sigma_rows, void* z_rows,
                                 tdg_stream stream);
tdg_status tdg_slab_unpack_z(tdg_plan p, int world, int rank, const void* recv, void* z_cols, tdg_stream stream);
tdg_status tdg_slab_columns(tdg_plan p, int world, int rank, const void* z_cols, void* g_cols, tdg_stream stream);
tdg_status tdg_slab_pack_g(tdg_plan p, int world, int rank, const void* g_cols, void* send, tdg_stream stream);
tdg_status tdg_slab_rows_inverse(tdg_plan p, int world, int rank, const void* g_rows, void* fx_rows,
                                 void* fy_rows, tdg_stream stream);

/* Transform lengths chosen for the plan: the padded periods px, py (even, 2^a 3^b,
 * >= 2n - 1) along x and y.  Any out pointer may be NULL. */
tdg_status tdg_plan_info(const tdg_plan p, int* px, int* py, int* order, int* precision);

/* Kernel path a forward solve of this plan runs: 0 = generic (any size, FP64 and FP32;
 * full spectra), 2 = FP32 one-barrier transform network (sides that are multiples of 16
 * from 128 to 4096 cells; half spectra in the network's order), 3 = the same network with
 * the column pass's DFT_16 stages on the tensor cores (the FP32_TC16 form).  Valid after
 * tdg_build_kernel_tables; -1 for a NULL plan. */
int tdg_plan_path(const tdg_plan p);

/* Release everything the plan owns (synchronises its device first). */
tdg_status tdg_destroy(tdg_plan p);

/* Static string naming a status code. */
const char* tdg_status_string(tdg_status s);

#ifdef __cplusplus
}
#endif

#endif /* TDGRAV_H */
