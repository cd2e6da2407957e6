/*
 * ps.h - periodic cubic-spline particle interpolation on one GPU (C ABI).
 *
 * The operations are those of Buaria & Yeung, "A highly scalable particle
 * tracking algorithm using PGAS programming for extreme-scale turbulence
 * simulations" (arXiv 2005.13193):
 *   Sec. 2.2, Operation 1  spline coefficients from the Eulerian field;
 *   Sec. 2.2, Operation 2  basis functions from particle positions;
 *   Sec. 2.2, Operation 3  64-term sum of Eq. (spline);
 *   Sec. 3                 particles handled where their stencil lives
 *                          (here: bin sort into cell bricks);
 *   Sec. 2.1 / 4.3         second-order Runge-Kutta particle advance.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every call returns a ps_status.  On failure ps_last_error() returns a
 *   thread-local message.  No C++ exception crosses this interface.
 * - Every GPU call is enqueued on `stream` (a cudaStream_t passed as void*;
 *   NULL = the legacy default stream) and returns before the GPU work ends.
 *   Argument errors are detected on the host before anything is enqueued.
 * - All array pointers are device pointers owned by the caller.  The library
 *   never frees them and, on these calls, allocates no device memory: scratch
 *   comes from the caller through (ws, ws_bytes), sized by the matching
 *   *_workspace_size() query.  ws must be 256-byte aligned.
 * - Device-side anomalies never trap: they are recorded in an optional
 *   caller-owned device word `int32_t status[4]` = {code, first index low 32
 *   bits, high 32 bits, count}.  A non-finite or out-of-range position gives
 *   NaN outputs for that particle (PS_DEV_NONFINITE_POS); a brick whose halo
 *   copy does not complete within the bounded wait (about a second) has its
 *   particles gather from global memory instead, so its outputs stay correct
 *   (PS_DEV_TIMEOUT).  Read it with ps_status_read().
 *
 * Layouts (x is the fastest index everywhere)
 * -------------------------------------------
 *   grid       n[0] = nx, n[1] = ny, n[2] = nz nodes on the periodic box
 *              [0,L[0]) x [0,L[1]) x [0,L[2]); node spacing h_d = L_d / n_d.
 *              3 <= n_d <= 2048.
 *   field      [ncomp][nz][ny][nx]                     (F32 or F64)
 *   coef       [ncomp][nz+3][ny+3][rx]                 (F32, F64, BF16, F16)
 *              padded index P in [0, n+2] holds node (P-1) mod n: one periodic
 *              ghost below and two above, the N+3 coefficients per line of
 *              Sec. 2.2.  Rows are padded to rx = ps_coef_row_pitch(nx, dtype)
 *              elements (nx+3 rounded up to 16 bytes; the tail is written as
 *              zero) so that every row starts on a 16-byte boundary.  Storage
 *              offset of (c, Pz, Py, Px) is ((c*(nz+3) + Pz)*(ny+3) + Py)*rx + Px.
 *              PS_F32X4: [nz+3][ny+3][nx+3][4] F32, node (Pz, Py, Px) holds
 *              (u, v, w, 0) at float offset ((Pz*(ny+3) + Py)*(nx+3) + Px)*4.
 *              (rx = nx+3 nodes.)
 *   scale      [ncomp][nz+3][ny+3] F32, only for BF16/F16 coefficients: the
 *              value of a coefficient is stored * scale of its x-line; scales
 *              are powers of two, so scaling itself is exact.
 *   pos        [3][np] FP64, structure of arrays; positions may lie outside
 *              the box (their periodic shadow image is used, Sec. 2.2).
 *   vel        [ncomp][np] F32.
 *   grad       [ncomp][3][np] F32, grad[c][d] = d u_c / d x_d.
 */
#ifndef PS_H
#define PS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PS_OK = 0,
  PS_ERR_INVALID_ARG = 1,   /* bad pointer, size, dtype or layout request   */
  PS_ERR_CUDA = 2,          /* a CUDA runtime call or kernel launch failed  */
  PS_ERR_WORKSPACE = 3,     /* ws NULL, misaligned or smaller than needed   */
  PS_ERR_UNSUPPORTED = 4,   /* valid request the library does not implement */
  PS_ERR_TIMEOUT = 5,       /* a bounded device wait gave up                */
  PS_ERR_DEVICE_STATUS = 6  /* ps_status_read found a device-side anomaly   */
} ps_status;

/* PS_F32X4 (coefficients only): the three components of a node stored
 * together as 16 bytes (u, v, w, 0); the array is [nz+3][ny+3][nx+3][4]
 * float, so one 16-byte load brings a node and a brick's halo is one box of
 * consecutive rows.  Requires ncomp == 3.  A storage choice, not part of the
 * method. */
/* PS_BF16X4 / PS_F16X4 (coefficients only): the same node layout with 16-bit
 * values (8 bytes per node, rows padded to an even node count), each scaled
 * by the power-of-two scale of its component's x-line; the scale array is
 * [nz+3][ny+3][4] F32 (s_u, s_v, s_w, 1).  The stored values are those of
 * PS_BF16 / PS_F16.  Requires ncomp == 3. */
typedef enum {
  PS_F32 = 0,
  PS_BF16 = 1,
  PS_F16 = 2,
  PS_F64 = 3,
  PS_F32X4 = 4,
  PS_BF16X4 = 5,
  PS_F16X4 = 6
} ps_dtype;

/* device status codes (status[0]) */
#define PS_DEV_OK 0
#define PS_DEV_NONFINITE_POS 1 /* position NaN/Inf or |x * n/L| >= 2^50 */
#define PS_DEV_TIMEOUT 2
#define PS_DEV_BAD_BINS 3 /* ps_rk2_step(rebin = 3) without the counts of a  */
                          /* preceding rebin = 2 or 3 step on the same ws   */

typedef struct {
  int32_t n[3]; /* nodes per axis: x, y, z */
  double L[3];  /* periodic box lengths (2*pi in the paper) */
} ps_grid;

/* Thread-local description of the last failure on this host thread. */
const char* ps_last_error(void);
/* Library version string. */
const char* ps_version(void);
/* Row pitch rx (elements) of a padded coefficient array for nx nodes along x:
 * nx+3 rounded up to a multiple of 16 bytes (PS_F32X4: nx+3 nodes of 16
 * bytes).  0 for a bad argument.  Part of
 * the storage layout, not of the method (the paper stores N+3 per line). */
int64_t ps_coef_row_pitch(int nx, ps_dtype coef_t);

/* Launch-shape knobs (not part of the method):
 *  "brick_kernel" (for the brick-staged calls, bins given): -1 = automatic
 *     (default; 5 for the gradient tensor and for 16-bit coefficients, 0
 *     otherwise), 0 = one CTA per brick, 8 lanes per particle, phases
 *     separated by block barriers, 2 = one CTA per brick, one thread per
 *     particle, 5 = one CTA per brick, four lanes per particle, each holding
 *     one z-row of the stencil in registers (the Heun predictor reuses it
 *     when it stays in its cell); 16-bit node halos stay 16-bit in shared
 *     memory.  Forms a case does not support fall back to 0.
 *  "brick_min_stage" in [0, 2^20] (default 8): bricks holding fewer particles
 *     skip the halo staging and gather their stencils from global memory.
 *  "node_tma" 0 or 1 (default 1): halos of node coefficients by tensor copy.
 *  "solve_xw" 0, 8, 16 or 32 (0 = default 16): x extent of a block of the
 *     strided spline passes.
 *  "solve_stream" 0 or 1 (default 1): FP32 solves in two streamed passes
 *     where they apply (ps_spline_coeffs).
 *  "solve_zt" 0, 16, 32, 64, 128 or 256 (0 = default: 256 planar, 64
 *     nodes): x columns per block of the streamed z pass.
 *  "solve_stages" 0, 2, 3 or 4 (0 = default 3): chunks in flight + 1 in the
 *     streamed x-y pass.
 *  "batch_run_below" in [0, 2^20] (default 16): ps_batch_plan bins a field
 *     whose bricks would hold fewer particles on average in runs of about
 *     128 neighbouring particles (stencils from global memory), not bricks.
 *  "batch_persistent" 0 or 1 (default 1): ps_batch_run runs all steps in one
 *     cooperative persistent launch (1) or a launch per phase and step (0).
 *  "wait_probe" in [0, 2^30] (default 0), a test knob: > 0 makes every
 *     staged brick wait, after its halo copy has landed, on a barrier that
 *     nothing completes, for that many clocks; the wait gives up, the status
 *     word reports PS_DEV_TIMEOUT and the brick's particles read their
 *     stencils from global memory (results unchanged).
 * Process-wide; set them before capturing work in a graph.  ps_tune_get
 * returns -1 for an unknown key (and for "brick_kernel" = automatic). */
ps_status ps_tune_set(const char* key, int64_t value);
int64_t ps_tune_get(const char* key);

/* Zero a device status word (4 x int32) on `stream`. */
ps_status ps_status_clear(int32_t* status, void* stream);
/* Copy a device status word to host_out[4], synchronising `stream`.
 * Returns PS_ERR_DEVICE_STATUS if host_out[0] != PS_DEV_OK. */
ps_status ps_status_read(const int32_t* status, int32_t* host_out, void* stream);

/* ------------------------------------------------------------------------ */
/* Operation 1 (Sec. 2.2): spline coefficients.                             */
/* Along every grid line of N nodes solve the periodic tridiagonal system   */
/* (1/6) c[j-1] + (4/6) c[j] + (1/6) c[j+1] = g[j] (indices mod N), for the */
/* x, y and z lines of every component, and store the N+3 padded           */
/* coefficients per axis.  The result is the exact inverse up to rounding;  */
/* the order of the three directions is immaterial in exact arithmetic.     */
/*   field_t: PS_F32 or PS_F64.  coef_t: PS_F32, PS_F64, PS_BF16, PS_F16,   */
/*   or the node forms PS_F32X4, PS_BF16X4, PS_F16X4 (ncomp == 3).          */
/*   Arithmetic is FP64 when coef_t is PS_F64, else FP32.                   */
/*   scale: required for BF16/F16 (per x-line power-of-two scale), else     */
/*   ignored.  field and coef must not overlap.  ncomp in [1, 16].          */
/*   ws: ps_spline_coeffs_workspace_size bytes, 256-byte aligned; required  */
/*   for the 16-bit and node forms.  For PS_F32 it is nonzero when nx is    */
/*   128, 256 or 512 and ny, nz >= 32: given it (and a 16-byte aligned F32  */
/*   field) the solve takes two streamed passes (x and y of every plane,    */
/*   then z), which truncate each periodic recursion's look-ahead at 16     */
/*   lines (terms below 7.2e-10 of the values skipped, under FP32           */
/*   rounding); without it the three passes run in place.  PS_F32X4 takes   */
/*   the two passes on the same grids.                                      */
/* ------------------------------------------------------------------------ */
size_t ps_spline_coeffs_workspace_size(const ps_grid* grid, int ncomp,
                                       ps_dtype coef_t);
ps_status ps_spline_coeffs(const ps_grid* grid, int ncomp, ps_dtype field_t,
                           const void* field, ps_dtype coef_t, void* coef,
                           float* scale, void* ws, size_t ws_bytes,
                           void* stream);

/* ------------------------------------------------------------------------ */
/* Operation 1 through the inverse (Sec. 2.2's periodic system, solved as a */
/* convolution): the inverse of the 1/6, 4/6, 1/6 circulant of N nodes has  */
/* entries G_N(d) = sqrt(3) (r^|d| + r^(N-|d|)) / (1 - r^N), r = sqrt(3)-2; */
/* keeping |d| <= K gives, along x, y and z,                                */
/*   c_j = sum_{d=-K..K} G_N(d) g_{(j+d) mod N},                            */
/* off the exact solve by less than 27 * 2 sqrt(3) |r|^(K+1) / (1 - |r|)    */
/* of max|g| (K = 15: 1e-7 relative, below FP32 rounding).  Every output    */
/* depends only on its 2K+1 neighbours per axis.                            */
/*   field: [ncomp][nz][ny][nx] F32, ncomp 1..3;  1 <= K <= 15, 2K+1 <= n.  */
/*   coef: the padded PS_F32 layout of ps_spline_coeffs ([ncomp][nz+3]     */
/*         [ny+3][rx], rx = ps_coef_row_pitch(nx, PS_F32)), 16-byte aligned.*/
/*   ws: ps_spline_truncated_workspace_size bytes, 256-byte aligned.        */
/* ------------------------------------------------------------------------ */
size_t ps_spline_truncated_workspace_size(const ps_grid* grid, int ncomp);
ps_status ps_spline_coeffs_truncated(const ps_grid* grid, int ncomp,
                                     const float* field, int K, float* coef,
                                     void* ws, size_t ws_bytes, void* stream);


/* ------------------------------------------------------------------------ */
/* Bin sort (Sec. 3: each particle is handled where the coefficients of its */
/* stencil live).  Cell a_d = floor(x_d * n_d/L_d) mod n_d (FP64, one       */
/* rounded multiply), brick b_d = a_d / brick[d], nb_d = ceil(n_d/brick[d]),*/
/* bin = (b_z*nb_y + b_y)*nb_x + b_x.  A counting sort gives                */
/*   bin_of[np]            int32 bin of each particle (required);           */
/*   bin_offsets[nbins+1]  int32 exclusive prefix sum of bin counts;        */
/*   perm[np]              int64 sorted slot -> particle index (optional);  */
/*   pos_sorted[3][np]     positions in sorted order (optional).            */
/* Within a bin the order is unspecified.  A non-finite position goes to    */
/* bin 0 and is flagged in `status` (optional).  np < 2^31.                 */
/* ------------------------------------------------------------------------ */
size_t ps_bin_workspace_size(const ps_grid* grid, const int32_t brick[3],
                             int64_t np);
ps_status ps_bin_particles(const ps_grid* grid, const int32_t brick[3],
                           int64_t np, const double* pos, int32_t* bin_of,
                           int32_t* bin_offsets, int64_t* perm,
                           double* pos_sorted, void* ws, size_t ws_bytes,
                           int32_t* status, void* stream);

/* ------------------------------------------------------------------------ */
/* ps_bin_particles without a workspace (no counterpart in the paper).      */
/* For callers that cannot allocate device memory or pass a workspace when  */
/* they bin: code under a device-memory budget owned by another allocator,  */
/* time-critical steps that must not add allocation latency, or plain C     */
/* hosts without an allocator of their own.  Same arguments, results and    */
/* errors as ps_bin_particles minus (ws, ws_bytes).  Nothing is allocated:  */
/* the counting-sort scratch lives in a fixed 32 MiB device array that      */
/* every GPU loading this library holds until the process exits; requests   */
/* needing more ((nbins + 1) + (nbins / 2048 + 2) + np int32 values, each   */
/* part rounded up to 256 bytes, above 32 MiB) fail with                    */
/* PS_ERR_INVALID_ARG before anything is enqueued.  The first call on a     */
/* device resolves the array's device address (cudaGetSymbolAddress) with   */
/* that device current: make it before any stream capture.  All calls share */
/* the one array (counters are cleared by each call), so calls that overlap */
/* on the GPU -- on different streams, or concurrent host threads -- race.  */
/* ------------------------------------------------------------------------ */
ps_status ps_bin_particles_noalloc(const ps_grid* grid, const int32_t brick[3],
                                   int64_t np, const double* pos,
                                   int32_t* bin_of, int32_t* bin_offsets,
                                   int64_t* perm, double* pos_sorted,
                                   int32_t* status, void* stream);

/* ------------------------------------------------------------------------ */
/* Operations 2 and 3 (Sec. 2.2, Eq. (spline)):                             */
/*   u_c(x) = sum_{i,j,k=0..3} b_i(t_x) b_j(t_y) b_k(t_z)                   */
/*            C_c[a_z+k][a_y+j][a_x+i]                                      */
/* with the uniform cubic B-spline b(t) = [(1-t)^3, 3t^3-6t^2+4,            */
/* -3t^3+3t^2+3t+1, t^3]/6 and t_d = x_d n_d/L_d - floor(x_d n_d/L_d).      */
/* FP64 positions, FP32 basis and accumulation (FP64 for PS_F64 coef).      */
/* Modes:                                                                   */
/*   bin_offsets == NULL             direct gather, any particle order;     */
/*   bin_offsets != NULL, perm NULL  particles stored in bin order (as left */
/*                                   by ps_bin_particles' pos_sorted or by  */
/*                                   ps_rk2_step); each brick's coefficient */
/*                                   halo is staged once in shared memory;  */
/*   bin_offsets and perm != NULL    same, particle perm[s] at sorted slot s.*/
/* brick[3] must be the one used for binning when bin_offsets != NULL.      */
/* Particles whose stencil leaves their brick's halo fall back to a direct  */
/* gather, so stale bins give correct (slower) results.                     */
/*   grad: optional [ncomp][3][np] velocity-gradient tensor.                */
/*   ncomp: 1 or 3.  status: optional.                                      */
/* ------------------------------------------------------------------------ */
ps_status ps_interp(const ps_grid* grid, int ncomp, ps_dtype coef_t,
                    const void* coef, const float* scale, int64_t np,
                    const double* pos, const int64_t* perm,
                    const int32_t* bin_offsets, const int32_t brick[3],
                    float* vel, float* grad, int32_t* status, void* stream);

/* ------------------------------------------------------------------------ */
/* Adjoint of ps_interp (and of ps_spline_coeffs) for a cotangent g_vel     */
/* [ncomp][np] F32:                                                         */
/*   g_pos[d][p]  = sum_c g_vel[c][p] d u_c / d x_d      ([3][np] FP64);    */
/*   g_field      = d <g_vel, u> / d field   ([ncomp][nz][ny][nx] F32):     */
/*                  scatter-add of g * basis weights, folded onto the N     */
/*                  periodic nodes (transpose of the padding), then the     */
/*                  same periodic solves (the matrix is symmetric).         */
/* Either output may be NULL.  g_field is overwritten (not accumulated).    */
/* Quantised (BF16/F16) coefficients are differentiated as if exact.        */
/* No workspace is needed (ws may be NULL with ws_bytes 0).                 */
/* ------------------------------------------------------------------------ */
ps_status ps_interp_backward(const ps_grid* grid, int ncomp, ps_dtype coef_t,
                             const void* coef, const float* scale, int64_t np,
                             const double* pos, const float* g_vel,
                             double* g_pos, float* g_field, void* ws,
                             size_t ws_bytes, int32_t* status, void* stream);

/* ------------------------------------------------------------------------ */
/* Second derivatives of the interpolant (the cubic spline is twice         */
/* continuously differentiable, Sec. 2.2): the 64-term sum of Eq. (spline)  */
/* with d2b/dt2 = (1-t, 3t-2, 1-3t, t) along one axis (or db/dt along two), */
/* times n_a n_b / (L_a L_b).                                               */
/*   perm, bin_offsets, brick: as for ps_interp.  bin_offsets == NULL:      */
/*   direct gathers, any particle order; given (three components, not      */
/*   F64): each brick's stencils from its halo staged in shared memory.     */
/*   hess: [ncomp][6][np] F32 in the order xx, yy, zz, xy, xz, yz.          */
/*   Non-finite positions give NaN and set the status word.                 */
/* ------------------------------------------------------------------------ */
ps_status ps_interp_hessian(const ps_grid* grid, int ncomp, ps_dtype coef_t,
                            const void* coef, const float* scale, int64_t np,
                            const double* pos, const int64_t* perm,
                            const int32_t* bin_offsets, const int32_t brick[3],
                            float* hess, int32_t* status, void* stream);

/* ------------------------------------------------------------------------ */
/* Lagrangian acceleration of fluid particles (Sec. 2.1: they move with the */
/* local velocity), a = du/dt + (u . grad) u, three components: the         */
/* convective term from the field at t (coef_n), du/dt as                   */
/* (u(coef_np1) - u(coef_n)) / dt_field when coef_np1 is given, else 0.     */
/*   acc: [3][np] F32; vel (optional): [3][np] F32, u from coef_n.          */
/*   dt_field > 0 when coef_np1 is given.  perm, bin_offsets, brick: as for */
/*   ps_interp (bin_offsets == NULL: direct gathers, any order; given: the  */
/*   stencils of coef_n from each brick's staged halo, those of coef_np1    */
/*   from global memory).                                                   */
/* ------------------------------------------------------------------------ */
ps_status ps_lagrangian_accel(const ps_grid* grid, ps_dtype coef_t,
                              const void* coef_n, const float* scale_n,
                              const void* coef_np1, const float* scale_np1,
                              double dt_field, int64_t np, const double* pos,
                              const int64_t* perm, const int32_t* bin_offsets,
                              const int32_t brick[3], float* acc, float* vel,
                              int32_t* status, void* stream);

/* ------------------------------------------------------------------------ */
/* One second-order Runge-Kutta step (Sec. 2.1; Sec. 4.3), Heun's form:     */
/*   u1 = u(x^n; coef_n);  x* = x^n + dt u1;  u2 = u(x*; coef_np1);         */
/*   x^{n+1} = x^n + (dt/2)(u1 + u2)                                        */
/* in FP64 for positions (velocities from the FP32 interpolation).          */
/* coef_np1 == NULL: frozen field (coef_n for both stages).  ncomp = 3.     */
/*   brick == NULL   particles keep their order; direct gathers.            */
/*   brick, rebin=1  particles are first bin-sorted by x^n and physically   */
/*                   reordered (pos, and ids if given), the analogue of the */
/*                   paper's particle migration (Sec. 4.3); bin_offsets     */
/*                   (optional, [nbins+1]) receives the new bin bounds;     */
/*                   stage 1 reads the staged brick halo in shared memory.  */
/*   brick, rebin=0  particles are taken to be in bin order already with    */
/*                   the given bin_offsets (required).  ws is optional:     */
/*                   when given, the step also counts the bins of the       */
/*                   positions it writes into ws, for a following           */
/*                   ps_rk2_sort(counted = 1) or ps_rk2_step(rebin = 3).    */
/*   brick, rebin=2  as rebin=1, and while it stores x^{n+1} the step       */
/*                   counts each particle's new bin into ws (bin, rank and  */
/*                   bin counters), the way the paper identifies departing  */
/*                   particles during the position update (Sec. 4.3).       */
/*   brick, rebin=3  as rebin=2, but the sort by x^n starts from the counts */
/*                   the previous rebin=2 or 3 call left in ws: that call   */
/*                   must have used the same grid, brick, np and ws, and    */
/*                   pos (and ids) must be as it left them.  The sort then  */
/*                   reads the positions once, not twice.  Counts that are  */
/*                   not those of pos are caught by range checks (each      */
/*                   write stays inside the arrays) and set PS_DEV_BAD_BINS */
/*                   in the status word.  Results equal rebin=1's, up to    */
/*                   the order of particles inside a bin.                   */
/*   vel_out: optional [3][np], receives u1 in the final particle order.    */
/*   ids: optional int64 [np] particle labels, permuted with the particles. */
/* ------------------------------------------------------------------------ */
size_t ps_rk2_workspace_size(const ps_grid* grid, const int32_t brick[3],
                             int64_t np);
ps_status ps_rk2_step(const ps_grid* grid, ps_dtype coef_t, const void* coef_n,
                      const void* coef_np1, const float* scale_n,
                      const float* scale_np1, int64_t np, double* pos,
                      int64_t* ids, float* vel_out, double dt,
                      const int32_t brick[3], int rebin, int32_t* bin_offsets,
                      void* ws, size_t ws_bytes, int32_t* status, void* stream);

/* ------------------------------------------------------------------------ */
/* The sort of a binned Heun step on its own (ps_rk2_step with rebin = 1    */
/* or 3 is this sort followed by the rebin = 0 step): particles pos [3][np] */
/* (and ids, optional int64 [np]) are copied in bin order to pos_sorted     */
/* (and ids_sorted; neither may alias its input) and bin_offsets           */
/* [nbins+1] receives the bin bounds.                                       */
/*   counted = 0: bins are counted from pos (as ps_bin_particles does);     */
/*   counted = 1: from the counts that the last ps_rk2_step on this ws      */
/*                (rebin = 0 with ws, 2 or 3) took of the positions it      */
/*                wrote, which pos must still hold; counts that are not     */
/*                pos's are caught by range checks and set PS_DEV_BAD_BINS. */
/* ws: ps_rk2_workspace_size(grid, brick, np) bytes, 256-byte aligned.      */
/* ------------------------------------------------------------------------ */
ps_status ps_rk2_sort(const ps_grid* grid, const int32_t brick[3], int64_t np,
                      const double* pos, const int64_t* ids, int counted,
                      double* pos_sorted, int64_t* ids_sorted,
                      int32_t* bin_offsets, void* ws, size_t ws_bytes,
                      int32_t* status, void* stream);

/* ------------------------------------------------------------------------ */
/* Many fields at once (no counterpart in the paper: a way of running many  */
/* of its problems together on one device).  A plan fixes the fields' grids */
/* and particle counts; particles of all fields live in one concatenated    */
/* [3][np_total] FP64 array, field f owning [base_f, base_{f+1})            */
/* (ps_batch_particle_base).  ps_batch_run optionally solves every field's  */
/* spline coefficients (solve = 1; ps_spline_coeffs per field), then takes  */
/* nsteps Heun steps of every particle (frozen fields): each step is one    */
/* bin sort over all particles (global bin = first bin of the field + bin   */
/* in the field) and one pass over the bricks of all fields, which counts  */
/* the next step's bins as it writes the positions (the first step counts   */
/* from the positions), all steps in one cooperative persistent launch      */
/* whose phases meet at grid-wide barriers (tune "batch_persistent" 0: a    */
/* launch per phase and step).  A                                           */
/* barrier wait that runs out (about 2^31 clocks) stops every block and     */
/* sets PS_DEV_TIMEOUT in *status; positions are then unspecified.          */
/* Particles end in bin order per field, as with ps_rk2_step(rebin=1); ids  */
/* (optional, int64 [np_total]) and vel_out (optional, [3][np_total] = u at */
/* the start of the last step) follow them.  use_graph = 1 captures the     */
/* solves and the steps in a CUDA graph on the first run and replays it     */
/* while the pointers, nsteps, dt and solve stay the same (the capture uses */
/* a stream owned by the plan; the graph is launched on `stream`).  The     */
/* plan holds host metadata, that stream and the graph; device scratch      */
/* comes from ws                                                            */
/* (ps_batch_workspace_size).  tune_cache: optional text file whose line    */
/* "brick <bx> <by> <bz>" overrides `brick` (written by the autotuner).     */
/* Coefficients: PS_F32, PS_BF16, PS_F16 or their node forms (PS_F32X4,    */
/* PS_BF16X4, PS_F16X4, whose halos are tensor copies); the batch uses the  */
/* one-CTA-per-brick kernel.                                                */
/* ------------------------------------------------------------------------ */
typedef struct ps_plan ps_plan;
typedef struct {
  const void* field; /* [3][nz][ny][nx] F32; read when solve = 1 */
  void* coef;        /* [3][nz+3][ny+3][rx] of coef_t (nodes: [nz+3][ny+3][rx][4]) */
  float* scale;      /* [3][nz+3][ny+3] for BF16/F16 ([nz+3][ny+3][4] for 16-bit */
                     /* nodes), else NULL */
} ps_batch_field;

ps_status ps_batch_plan(int nfields, const ps_grid* grids, const int64_t* nps,
                        ps_dtype coef_t, const int32_t brick[3],
                        const char* tune_cache, ps_plan** out);
size_t ps_batch_workspace_size(const ps_plan* plan);
int64_t ps_batch_num_particles(const ps_plan* plan);
/* First particle of field `field` (field = nfields gives np_total). */
int64_t ps_batch_particle_base(const ps_plan* plan, int field);
ps_status ps_batch_run(ps_plan* plan, const ps_batch_field* fields, int solve,
                       double* pos, int64_t* ids, float* vel_out, int nsteps,
                       double dt, int use_graph, void* ws, size_t ws_bytes,
                       int32_t* status, void* stream);
void ps_plan_destroy(ps_plan* plan);

#ifdef __cplusplus
}
#endif

#endif /* PS_H */
