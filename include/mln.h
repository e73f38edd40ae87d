/*
 * mln.h -- C-ABI of the GB300 (sm_103a) Maxwell-Liouville-von Neumann solver.
 *
 * The library advances the one-dimensional Maxwell-Liouville-von Neumann
 * (MLN) equations of Riesch & Jirauschek (arXiv:1710.09799):
 *   - Maxwell's curl equations for E_z and H_y with the polarisation current
 *     dP/dt as source (Sec. 2, Eq. 1), on the staggered FDTD grid of Fig. 1;
 *   - the Liouville-von Neumann equation of every medium cell in the adjoint
 *     (SU(N), pseudospin) representation, d/dt d = (M + U E_z) d + d_eq
 *     (Sec. 3, Eq. 14), advanced by the symmetric Strang splitting of
 *     Sec. 4.1 (Eq. 23) with the interaction exponential exp(U E_z dt) done by
 *     the diagonalisation method of Sec. 4.2 (Eq. 25) in its real form
 *     (the matrix T of Eq. 26): per cell only scalar sin/cos and small dense
 *     products;
 *   - dP/dt = N_a/2 v^T (M d + d_eq) (Sec. 3, Eq. 17).
 * One time step: H^{n+1/2} from E^n; d^{n-1/2} -> d^{n+1/2} with E^n;
 * dP/dt^{n+1/2}; E^{n+1} from H^{n+1/2} and dP/dt^{n+1/2}; then the source.
 *
 * Conventions for every call:
 *   - All entry points return an mln_status; no exception crosses the ABI.
 *     The context keeps a message with details (mln_last_error).
 *   - Complex matrices are arrays of interleaved (re, im) doubles, row-major.
 *     A superoperator is an (N*N) x (N*N) complex matrix acting on the
 *     row-major vectorisation vec(X)[j*N + k] = X[j][k].
 *   - Units are SI: J, C*m, 1/s, V/m, A/m, m, s.
 *   - Device buffers passed to mln_create are owned by the caller and must
 *     outlive the context. The context owns a second copy of the state (the
 *     steps alternate between the two), a few hundred bytes of flags and the
 *     output conversion tables; mln_destroy frees them.
 *   - Work is queued on the CUDA stream given at creation. Calls that return
 *     data to the host synchronise that stream.
 */
#ifndef MLN_H
#define MLN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum mln_status {
    MLN_OK = 0,
    MLN_EINVAL = 1,        /* invalid argument or parameter set */
    MLN_ENOMEM = 2,        /* host or device allocation failed */
    MLN_ECUDA = 3,         /* a CUDA runtime call failed */
    MLN_ENUMERIC = 4,      /* host set-up failed a numerical check */
    MLN_ETIMEOUT = 5,      /* a bounded device wait gave up */
    MLN_EUNSUPPORTED = 6,  /* valid but not built (e.g. N outside the compiled range) */
    MLN_ENONFINITE = 7     /* the device saw a non-finite field value */
} mln_status;

enum { MLN_BC_PERIODIC = 0, MLN_BC_OPEN = 1 };
enum { MLN_SRC_NONE = 0, MLN_SRC_HARD = 1, MLN_SRC_SOFT = 2 };
enum { MLN_FP64 = 0, MLN_FP32 = 1 };
/* MLN_FORM_STRANG applies the three updates of Eq. 23 as written: half a
 * step of exp(M dt/2), the interaction exp(U E dt) through the eigenbasis T,
 * half a step of exp(M dt/2).
 * MLN_FORM_MERGED fuses the second half-step of one step with the first
 * half-step of the next into one affine map (A0^2, A0 b + b); the state is
 * then the vector after the first half-step. Same result up to rounding,
 * three D x D products per step instead of four.
 * Both apply each propagator as identity + increment, which keeps the
 * rounding of the small coherences at their own scale. */
/* MLN_FORM_RODRIGUES (N <= 4) is the literal Strang form with the interaction
 * exponential evaluated by the generalised Rodrigues formula of Eq. 27,
 * I + sum_k sin(a_k) S_k + (1 - cos a_k) S_k^2, with the rank-2 matrices
 * S_k = T Theta_k T^T (and S_k^2) stored in full: the paper's "rodr" method. */
/* MLN_FORM_ROTATED is the merged form with the state held in the basis of
 * the rotation planes, z = T^T y: a step rotates the plane pairs of z by the
 * angles of Eq. 24 and applies one affine map C z'' + c' with
 * C = T^T A0^2 T and c' = T^T (A0 b + b), and dP/dt = (T^T A0^T w) . z'' +
 * w . b + c. One dense D x D product per step instead of the merged form's
 * three (T^T, T and A0^2 - I): fewer operations where T is dense (N >= 5;
 * the six-level model: 2750 against 6919 flops per cell update), more where
 * T is sparse and C is not (the three-level ring: 199 against 179). Same
 * result up to rounding. Runs on the run-time compiled kernel
 * (MLN_KERNEL_JIT; in FP64 also in double-float pairs, MLN_KERNEL_DF32) or,
 * in FP32 with N = 5 or 6, on the tensor cores
 * (MLN_KERNEL_TENSOR, which MLN_KERNEL_AUTO picks there), with the FDTD field
 * solver, single grids (no batches, adjoint or allocation-free step). */
enum { MLN_FORM_STRANG = 0, MLN_FORM_MERGED = 1, MLN_FORM_RODRIGUES = 2, MLN_FORM_ROTATED = 3 };
/* Cell model of the step kernel. MLN_KERNEL_REGISTER keeps each cell's
 * vector in registers and multiplies by the full D x D constant matrices.
 * MLN_KERNEL_SPARSE (FP64, merged form only) keeps the vectors in shared
 * memory and multiplies only by the entries of the constant matrices that
 * are not exactly zero; the sums run in the same order, so both give the
 * same result. MLN_KERNEL_AUTO picks TENSOR for FP32 merged or rotated with
 * N = 5 or 6 (the dense case); JIT for the other merged FDTD problems (FP64
 * and FP32) when NVRTC is available and for the other rotated-basis problems;
 * SPARSE for FP64 merged problems otherwise (without NVRTC, or with the PSTD
 * field solver); REGISTER otherwise. */
/* MLN_KERNEL_JIT (merged form) generates, at mln_create, this problem's step
 * as straight-line CUDA with the constants as literals and the exactly-zero
 * entries left out, compiles it for sm_103a at run time (NVRTC) and launches
 * it; same arithmetic and order as MLN_KERNEL_REGISTER, so the same bits.
 * It needs libnvrtc at run time (MLN_EUNSUPPORTED otherwise). */
/* MLN_KERNEL_TENSOR (FP32, merged or rotated form, N = 5 or 6) runs the
 * dense products of a step on the fifth-generation tensor cores (tcgen05.mma,
 * 128 cells per MMA, accumulators in tensor memory). Merged form
 * (kind::tf32): two products per step (the plane coordinates T^T y, then the
 * increment of y and dP/dt from [y ; dz] in one product), each FP32 operand
 * split into a high and a low TF32 part. Rotated form (kind::f16): one
 * product per step (the increment of z and dP/dt from [z'' ; 1]), each
 * operand scaled by powers of two and split into a high and a low FP16 part.
 * Three MMAs per K block in both (hi*hi, hi*lo, lo*hi): FP32-level accuracy,
 * not the FP32 register model's bits. Up to 32 steps per launch (block_steps;
 * larger values are an error with MLN_KERNEL_TENSOR and are capped at 32 when
 * MLN_KERNEL_AUTO picks it), tiles of 128 - 2 block_steps cells; tile_cells is
 * ignored. */
/* MLN_KERNEL_DF32 (MLN_FP64, merged form or rotated basis, FDTD) is the run-time
 * compiled step of MLN_KERNEL_JIT in double-float arithmetic (also for the
 * grids of a batch, mln_batch_create): every value of
 * the step (the cell update's products, plane rotation and dP/dt, and the
 * E and H update) a pair of FP32 numbers h + l, about 48 significant bits,
 * on the FP32 pipe, whose throughput is 64 times the FP64 pipe's. The state,
 * E and H stay FP64 in memory, converted at the start and end of each launch.
 * Not the FP64 bits, and the rounding of the pairs (2^-48 against 2^-53)
 * adds up in the field recurrence: against the FP64 oracle, E_z within
 * 9e-13 on the three-level ring after 1500 steps, 5e-11 on the two-level
 * grid after 20000 steps, on a six-level grid (D = 35) after 400 1.1e-10
 * (merged form) and 5e-11 (rotated basis, blocks of at most 256 threads).
 * Rotation angles above 2^-12 are evaluated in FP64. MLN_EUNSUPPORTED
 * without NVRTC or when a constant of the step lies outside the pair's range
 * (above 1e37, or non-zero below 1e-30 in magnitude). Never chosen by
 * MLN_KERNEL_AUTO. */
enum {
    MLN_KERNEL_AUTO = 0,
    MLN_KERNEL_REGISTER = 1,
    MLN_KERNEL_SPARSE = 2,
    MLN_KERNEL_JIT = 3,
    MLN_KERNEL_TENSOR = 4,
    MLN_KERNEL_DF32 = 5
};

/* Field solver (mln_params.maxwell). MLN_MAXWELL_FDTD: the staggered finite
 * differences of the paper's Fig. 1, fused with the medium update and
 * temporal blocking. MLN_MAXWELL_PSTD: the pseudo-spectral variant that the
 * paper's Secs. 1 and 3 say the method carries over to: on a periodic grid,
 * dE_z/dx at the H_y points and dH_y/dx at the E_z points are the derivatives
 * of the trigonometric interpolant of the samples (FFT, multiplier
 * i k e^{+-i k dx/2}); the time stepping and the medium step are unchanged.
 * PSTD needs MLN_BC_PERIODIC, n_cells a power of two in [16, 2^24], and
 * kernel MLN_KERNEL_AUTO, MLN_KERNEL_REGISTER or MLN_KERNEL_SPARSE (AUTO picks
 * SPARSE for FP64 merged problems, REGISTER otherwise). Each step is several
 * kernel launches (the medium, then the FFT passes of the two derivatives);
 * it runs in place on the caller's buffers. Batches, mln_adjoint and
 * mln_step_noalloc take FDTD problems only. */
enum {
    MLN_MAXWELL_FDTD = 0,
    MLN_MAXWELL_PSTD = 1
};

#define MLN_MIN_N 2
#define MLN_MAX_N 6

/*
 * Problem description. Every pointer is read during mln_create only.
 *   N             number of levels, MLN_MIN_N..MLN_MAX_N; adjoint dimension D = N*N-1.
 *   precision     MLN_FP64 or MLN_FP32: type of the device state, fields and
 *                 propagator arithmetic. Set-up is always FP64.
 *   form          MLN_FORM_STRANG, MLN_FORM_MERGED, MLN_FORM_RODRIGUES (N <= 4)
 *                 or MLN_FORM_ROTATED (run-time compiled kernel, FDTD).
 *   H0            N x N complex Hermitian, J (Eq. 2, H = H0 - mu E_z).
 *   mu            N x N complex Hermitian dipole operator, C m.
 *   G             (N*N) x (N*N) complex relaxation superoperator, 1/s; it must
 *                 preserve trace and Hermiticity (Eq. 2). NULL: no relaxation.
 *   rho0          N x N complex initial density matrix of every medium cell:
 *                 Hermitian, unit trace, positive semidefinite.
 *   N_a           density of quantum systems, m^-3 (Eq. 3).
 *   n_cells       number of E_z cells (>= 4).
 *   medium_begin, medium_end  the medium occupies cells [begin, end).
 *   dx, dt        grid spacing (m) and time step (s); c dt / dx <= 1.
 *   eps_r, mu_r, sigma  relative permittivity and permeability (> 0) and
 *                 conductivity (>= 0, S/m) of the whole grid (Eq. 1).
 *   boundary      MLN_BC_PERIODIC: ring. MLN_BC_OPEN: E_z at cell 0 changes
 *                 only through a hard source at cell 0, the right end uses the
 *                 first-order Mur absorbing condition; the medium must end at
 *                 least one cell before the last cell.
 *   source_kind, source_cell  MLN_SRC_HARD replaces, MLN_SRC_SOFT adds the
 *                 sample to E_z at source_cell after the E_z update; sample k
 *                 of an mln_step call belongs to the step producing E^{n+1},
 *                 n = the context's step count at the call + k.
 *   block_steps   steps fused into one kernel launch (temporal blocking);
 *                 0 picks a default. 1..64.
 *   tile_cells    cells written by one thread block; 0 picks a default.
 *   kernel        MLN_KERNEL_AUTO, MLN_KERNEL_REGISTER, MLN_KERNEL_SPARSE,
 *                 MLN_KERNEL_JIT, MLN_KERNEL_TENSOR or MLN_KERNEL_DF32.
 *   maxwell       MLN_MAXWELL_FDTD (0) or MLN_MAXWELL_PSTD.
 */
typedef struct mln_params {
    int32_t N;
    int32_t precision;
    int32_t form;
    int32_t boundary;
    int32_t source_kind;
    int32_t block_steps;
    int32_t tile_cells;
    int32_t kernel;
    const double *H0;
    const double *mu;
    const double *G;
    const double *rho0;
    double N_a;
    int64_t n_cells;
    int64_t medium_begin;
    int64_t medium_end;
    int64_t source_cell;
    double dx;
    double dt;
    double eps_r;
    double mu_r;
    double sigma;
    int32_t maxwell;
} mln_params;

typedef struct mln_ctx mln_ctx;

/*
 * Sizes of the caller-owned device buffers for a parameter set:
 *   state_bytes  the per-cell state of the medium, structure of arrays:
 *                element j of medium cell m (cell medium_begin + m) is at
 *                index j * stride + m, j < D, stride = n_medium rounded up to
 *                a multiple of 64; real type = precision.
 *   field_bytes  one of E_z or H_y: n_cells reals (H_y[i] sits at i + 1/2).
 * Returns MLN_EINVAL for an invalid parameter set (same checks as mln_create).
 */
mln_status mln_query_buffers(const mln_params *p, size_t *state_bytes, size_t *field_bytes);

/*
 * Validate p, compute the FP64 set-up of Secs. 3-4 (generators, M, U, d_eq,
 * v, A0 = exp(M dt/2) with its affine offset, the real eigenbasis T and
 * rotation rates of U, polarisation coefficients), allocate the context's
 * alternate state, and queue on `stream` (a cudaStream_t; NULL = legacy
 * default stream) the initial medium state built from rho0 into d_state.
 * Ez and Hy are used as they are: the caller fills them with E^0 and
 * H^{-1/2} (zeros, noise, ...). d_state, Ez and Hy are device pointers with
 * the sizes of mln_query_buffers, 16-byte aligned.
 * Errors: MLN_EINVAL (bad parameters: N range, Hermiticity to 1e-12
 * relative, rho0 trace/positivity, G trace/Hermiticity preservation, ranges,
 * dt, Courant number), MLN_ENUMERIC (eigen-decomposition residual above
 * 1e-12), MLN_EUNSUPPORTED, MLN_ENOMEM, MLN_ECUDA. On error *out is NULL.
 */
mln_status mln_create(const mln_params *p, void *d_state, void *Ez, void *Hy, void *stream,
                      mln_ctx **out);

/*
 * Queue n_steps time steps (>= 0) on the context's stream. src is NULL (no
 * source) or a device array of n_steps doubles (see source_kind). When the
 * call returns, the queued work leaves the current state in the caller's
 * buffers. Device-side problems (non-finite E_z) are reported by the next
 * mln_sync or read call.
 */
mln_status mln_step(mln_ctx *ctx, int64_t n_steps, const double *src);

/*
 * Positivity projection of the medium state (optional; FP64 on the device, off
 * the step path). Trace and Hermiticity of every cell's rho hold by
 * construction in the adjoint representation (Eq. 6); rounding (most of all
 * in FP32) can leave rho with a slightly negative eigenvalue. For each such
 * cell this replaces rho by the nearest positive semidefinite unit-trace
 * matrix in the Frobenius norm (eigenvalues projected onto the probability
 * simplex, eigenvectors kept; Hermitian eigen-decomposition by complex Jacobi
 * rotations). Cells whose smallest eigenvalue is at least -16 N u (u = 2^-53
 * in FP64, 2^-24 in FP32: a zero eigenvalue after rounding) keep their state
 * bit for bit. Queued on the context's stream after the work already there;
 * synchronous.
 *   n_projected  NULL or receives the number of cells changed.
 * Call it every K steps for a periodic re-projection.
 */
mln_status mln_project_positive(mln_ctx *ctx, int64_t *n_projected);

/* Wait for the queued work; report device-side problems (MLN_ENONFINITE, or
 * MLN_ETIMEOUT when a tensor-core kernel gave up waiting for an MMA). */
mln_status mln_sync(mln_ctx *ctx);

/* Number of time steps taken so far. */
int64_t mln_step_count(const mln_ctx *ctx);

/* Number of fused-step kernel launches queued so far, and the launch shape
 * in use: steps fused per launch and cells written per thread block. */
int64_t mln_launch_count(const mln_ctx *ctx);
/* The cell model the context's step kernel uses (MLN_KERNEL_REGISTER,
 * MLN_KERNEL_SPARSE, MLN_KERNEL_JIT, MLN_KERNEL_TENSOR or MLN_KERNEL_DF32),
 * -1 for NULL. */
int32_t mln_kernel_in_use(const mln_ctx *ctx);
mln_status mln_launch_shape(const mln_ctx *ctx, int32_t *block_steps, int32_t *tile_cells,
                            int32_t *threads_per_block);

/*
 * Autotuner: time candidate launch shapes (steps fused per launch K and cells
 * per thread block) on this context and keep the fastest. Each candidate is
 * timed by repeating one launch that reads the caller's buffers and writes
 * the context's alternate copy, so the state is not changed. trials: timed
 * launches per candidate (>= 1). The chosen K and tile are returned (either
 * pointer may be NULL) and used by later mln_step calls. Synchronises.
 */
mln_status mln_autotune(mln_ctx *ctx, int32_t trials, int32_t *block_steps, int32_t *tile_cells);

/*
 * Algorithmic work of one time step, for roofline accounting (not a
 * measurement): flops_medium = flops (FMA = 2, other operations 1) of one
 * medium cell-update, counting only the entries of the constant matrices that
 * are not exactly zero and only the rotation-plane columns of T (the work the
 * method needs for this problem, whatever the cell model executes), with the
 * shortest series for (sin, cos - 1); flops_cell = flops of the FDTD updates
 * of one grid cell (9); bytes_medium / bytes_cell = device-memory bytes one
 * launch reads and writes per medium / vacuum cell (state and fields, once
 * each way). Any output pointer may be NULL.
 */
mln_status mln_work_per_step(const mln_ctx *ctx, double *flops_medium, double *flops_cell, double *bytes_medium,
                             double *bytes_cell);

/*
 * Copy E_z^n and H_y^{n-1/2} (n = step count) to host arrays of n_cells
 * doubles each (either may be NULL). Synchronises.
 */
mln_status mln_get_fields(mln_ctx *ctx, double *Ez_host, double *Hy_host);

/*
 * Density matrices rho^{n-1/2} of medium cells [cell0, cell0 + count) (grid
 * cell indices) into rho_host, count * N * N complex, converted on the device
 * by rho = I/N + 1/2 sum_j d_j s_j (Eq. 6). Synchronises.
 */
mln_status mln_get_rho(mln_ctx *ctx, int64_t cell0, int64_t count, double *rho_host);

/* Populations rho_ll of medium cells [cell0, cell0 + count): count * N doubles. */
mln_status mln_get_populations(mln_ctx *ctx, int64_t cell0, int64_t count, double *pop_host);

/*
 * Checkpoint / resume in a precision- and form-independent layout:
 * d_host holds n_medium * D doubles, cell-major (d of medium cell m at
 * m * D .. m * D + D - 1, adjoint vector of Eq. 6), Ez_host and Hy_host
 * n_cells doubles each. Either call may take NULL for parts it should skip.
 * save synchronises; load queues the host-to-device copies on the stream and
 * returns after they are complete.
 */
mln_status mln_save_state(mln_ctx *ctx, double *d_host, double *Ez_host, double *Hy_host);
mln_status mln_load_state(mln_ctx *ctx, const double *d_host, const double *Ez_host,
                          const double *Hy_host);

/*
 * Adjoint gradients (reverse-time, discrete adjoint of the literal Strang
 * step of Eq. 23 with the FDTD update of Eq. 1, boundaries and source included).
 * Objective J = dt * sum_{n=1..n_steps} (E_z^n at probe_cell)^2, the field
 * energy density at an output cell integrated over the run, starting from the
 * context's current state; the context ends advanced by n_steps (by its own
 * form and cell model). Any form: the forward pass runs the context's step and
 * checkpoints its state; each segment is recomputed, from the checkpoint
 * mapped to the adjoint vector d, in the Strang form, which all forms equal up
 * to rounding, and differentiated there. Periodic rings and open grids (held
 * cell 0 with a hard or soft source, Mur at the right end). Needs N <= 4 and
 * MLN_MAXWELL_FDTD (MLN_EUNSUPPORTED otherwise).
 *   src         as for mln_step (device, n_steps samples) or NULL.
 *   every       checkpoint interval: the forward pass saves the state every
 *               `every` steps; the backward pass recomputes each segment from
 *               its checkpoint, keeping each step's state, fields and traced
 *               intermediates (a "set", about 3 x the state bytes). When the
 *               sets of all segments (about n_steps + n_steps / every of them)
 *               fit the memory limit (mln_set_adjoint_memory), a Strang-form
 *               context on the register model records them in its forward
 *               pass (nothing recomputed) and any other context recomputes
 *               every segment at once, side by side, after its forward pass;
 *               the backward pass then runs from one CUDA graph captured on
 *               a stream of the call's own. Otherwise two segments' sets are
 *               kept and segment s - 1 is recomputed while the reverse sweep
 *               of segment s runs. All give the same bits.
 *   out->J      the objective.
 *   out->dJ_dsrc  NULL or n_steps doubles: dJ / d(source sample k).
 *   out->dJ_dmu   NULL or N*N doubles: dJ / d mu_ll (l = 0..N-1), then
 *               dJ / d Re mu_jk, then dJ / d Im mu_jk for j < k in row-major
 *               order (mu_kj follows as the conjugate). The eigenvalues of mu
 *               must be distinct (MLN_ENUMERIC otherwise).
 *   out->dJ_dG    NULL or (N*N)^2 complex (interleaved): Gamma with
 *               dJ = Re sum_rc conj(Gamma_rc) dG_rc for the relaxation
 *               superoperator of the parameter set (zero rows and columns included).
 * Device memory for the checkpoints, the recorded sets and the adjoints is one
 * workspace that the context keeps after the call and reuses in its next
 * mln_adjoint call when it is large enough (else it is freed and a larger one
 * allocated); mln_adjoint_release or mln_destroy frees it. Synchronises.
 *
 * mln_set_adjoint_memory: the most device memory, in bytes, that mln_adjoint
 * on this context may take for the recorded sets of all segments at once;
 * 0 (the default): half of the free device memory at the call plus the
 * workspace the context already holds. MLN_EINVAL for a negative value.
 *
 * mln_adjoint_release: wait for the context's stream, then free the adjoint
 * workspace it holds (nothing to do if it holds none). MLN_EINVAL for NULL,
 * MLN_ECUDA if the wait or the free fails.
 */
typedef struct mln_adjoint_out {
    double J;
    double *dJ_dsrc;
    double *dJ_dmu;
    double *dJ_dG;
} mln_adjoint_out;
mln_status mln_set_adjoint_memory(mln_ctx *ctx, int64_t bytes);
mln_status mln_adjoint_release(mln_ctx *ctx);
mln_status mln_adjoint(mln_ctx *ctx, int64_t n_steps, const double *src, int64_t probe_cell, int32_t every,
                       mln_adjoint_out *out);

/*
 * Batches: many independent grids advanced together. Every K steps, one
 * launch per N present covers every tile of every grid with that N (a kernel
 * compiled for each N, so each gets the registers of its own cell size), so
 * small and large grids share the GPU; the launches of one mln_batch_step
 * call are captured into a CUDA graph and replayed as one graph launch.
 *
 * mln_batch_create: count grids, params[i] as for mln_create with one common
 * precision, form MLN_FORM_MERGED, N <= 4 and kernel AUTO, REGISTER or JIT,
 * or MLN_KERNEL_DF32 with MLN_FP64 for every grid (the batch kernels in
 * double-float pairs, each grid's constants staged as pairs);
 * d_state[i], Ez[i], Hy[i] caller-owned device buffers as for mln_create;
 * src NULL or count device pointers to src_len source samples per grid
 * (sample k applies to the batch's step k; NULL entries for grids without a
 * source); stream as for mln_create. Each grid gets an internal context
 * (alternate buffers, tables). Errors as mln_create, message in
 * mln_create_error().
 * mln_batch_autotune: choose steps per launch and tile size (same for every
 * grid) by timing candidates that read the caller's buffers and write the
 * contexts' own, so the state is not changed. Synchronises.
 * mln_batch_step: queue n_steps steps of every grid (async, one graph launch
 * on the batch's own stream, ordered after the work already queued on the
 * creation stream, which in turn waits for the graph).
 * mln_batch_sync: wait; read and clear every grid's device-side flags and report the
 * first grid's problem.
 * mln_batch_context: the internal context of grid i, for reading results
 * (mln_get_fields, mln_get_rho, mln_save_state, ...); owned by the batch:
 * do not step or destroy it.
 * mln_batch_shape: steps per launch, tile, work items (tiles of every grid,
 * over the per-N launches of one step of K), kernel launches queued so far.
 * mln_batch_error: message of the last failed call on the batch.
 * mln_batch_kernel_in_use: the cell model of the batch's N-level grids:
 * MLN_KERNEL_JIT (a kernel compiled at mln_batch_create for the union of the
 * non-zero entries of those grids' constant matrices, each grid's constants
 * staged in shared memory and, when they fit, held in registers; the default
 * when NVRTC is available and no grid asks for MLN_KERNEL_REGISTER) or
 * MLN_KERNEL_REGISTER (dense products, padded constants in shared memory);
 * both give the register model's bits; or MLN_KERNEL_DF32 for a batch of
 * double-float grids (the bits of those grids stepped alone at the same
 * steps per launch); -1 if the batch has no grid with N levels.
 * mln_batch_kernel_source: host only; the CUDA source that the batch with
 * these params would compile for its N-level grids (as mln_kernel_source).
 * mln_batch_set_launch: the launch structure of later mln_batch_step calls.
 * MLN_BATCH_CHUNKS (the default): one launch per K steps and N, as above.
 * MLN_BATCH_PERSISTENT: one launch per call and N; its blocks take (chunk,
 * tile) items in chunk-major order from a device counter and, before chunk c
 * of a tile, wait until the tiles within halo + 1 cells of it have completed
 * chunk c - 1 (per-tile progress counters). Same arithmetic, same bits as the
 * chunked launches. Each wait polls at most wait_limit times (100 ns apart);
 * a wait that gives up sets a flag, the kernel carries on, and the next
 * mln_batch_sync returns MLN_ETIMEOUT (wait_limit 0 gives up at once: a test
 * of that path). Needs the run-time compiled batch kernels (every N of the
 * batch on MLN_KERNEL_JIT) and tiles of at least K + 2 cells (what
 * mln_batch_autotune chooses); MLN_EUNSUPPORTED otherwise, MLN_EINVAL for an
 * unknown mode or a negative limit. Synchronises the batch's stream and
 * drops its captured graphs.
 * mln_batch_launch: the launch structure of the next mln_batch_step (-1 for
 * a NULL batch).
 */
typedef struct mln_batch mln_batch;
mln_status mln_batch_create(int32_t count, const mln_params *params, void *const *d_state, void *const *Ez,
                            void *const *Hy, const double *const *src, int64_t src_len, void *stream,
                            mln_batch **out);
mln_status mln_batch_autotune(mln_batch *b, int32_t trials, int32_t *block_steps, int32_t *tile_cells);
mln_status mln_batch_step(mln_batch *b, int64_t n_steps);
mln_status mln_batch_sync(mln_batch *b);
mln_ctx *mln_batch_context(mln_batch *b, int32_t i);
mln_status mln_batch_shape(const mln_batch *b, int32_t *block_steps, int32_t *tile_cells, int64_t *items,
                           int64_t *launches);
const char *mln_batch_error(const mln_batch *b);
int32_t mln_batch_kernel_in_use(const mln_batch *b, int32_t N);
mln_status mln_batch_kernel_source(int32_t count, const mln_params *params, int32_t N, char *buf, size_t cap,
                                   size_t *len);
enum { MLN_BATCH_CHUNKS = 0, MLN_BATCH_PERSISTENT = 1 };
mln_status mln_batch_set_launch(mln_batch *b, int32_t mode, int32_t wait_limit);
int32_t mln_batch_launch(const mln_batch *b);
void mln_batch_destroy(mln_batch *b);

/* Free the context (NULL-safe). Caller buffers are not touched. */
void mln_destroy(mln_ctx *ctx);

const char *mln_status_string(mln_status s);
/* Last error message of a context (empty string if none; "" for NULL). */
const char *mln_last_error(const mln_ctx *ctx);
/* Last error message of a failed mln_create, mln_setup_host, mln_query_buffers
 * or mln_step_noalloc on this thread. */
const char *mln_create_error(void);

/*
 * Host-only inspection of the FP64 set-up (no GPU needed). Arrays are
 * row-major doubles with the sizes given; the caller provides capacity for
 * D_max = MLN_MAX_N^2 - 1.
 *   M, U, A0, T, C1 (= A0^2 - I): D x D;  d_eq, v, b, w, d0: D;
 *   theta: q = N(N-1)/2 rotation rates (rad s^-1 per V/m: plane k of T turns
 *   by theta_k E dt in a step); c: scalar; gen: D x N x N complex generators
 *   (2 * D * N * N doubles, Sec. 3 ordering u_jk, v_jk, w_l).
 */
typedef struct mln_setup {
    int32_t N, D, q, reserved;
    double M[(MLN_MAX_N * MLN_MAX_N - 1) * (MLN_MAX_N * MLN_MAX_N - 1)];
    double U[(MLN_MAX_N * MLN_MAX_N - 1) * (MLN_MAX_N * MLN_MAX_N - 1)];
    double A0[(MLN_MAX_N * MLN_MAX_N - 1) * (MLN_MAX_N * MLN_MAX_N - 1)];
    double T[(MLN_MAX_N * MLN_MAX_N - 1) * (MLN_MAX_N * MLN_MAX_N - 1)];
    double C1[(MLN_MAX_N * MLN_MAX_N - 1) * (MLN_MAX_N * MLN_MAX_N - 1)];
    double d_eq[MLN_MAX_N * MLN_MAX_N - 1];
    double v[MLN_MAX_N * MLN_MAX_N - 1];
    double b[MLN_MAX_N * MLN_MAX_N - 1];
    double w[MLN_MAX_N * MLN_MAX_N - 1];
    double d0[MLN_MAX_N * MLN_MAX_N - 1];
    double theta[MLN_MAX_N * (MLN_MAX_N - 1) / 2];
    double c;
    double gen[2 * (MLN_MAX_N * MLN_MAX_N - 1) * MLN_MAX_N * MLN_MAX_N];
} mln_setup;

mln_status mln_setup_host(const mln_params *p, mln_setup *out);

/*
 * Host-only helper: the relaxation superoperator of a Lindblad dissipator
 * with jump operators L = |a><b| (level b decays to level a at rate
 * gamma_{b->a}) plus pure dephasing of the coherences (the linear relaxation
 * term of Eq. 2, written in the form the G parameter takes):
 *   G(rho) = sum_{a,b} gamma_{b->a} (L rho L^+ - (L^+ L rho + rho L^+ L) / 2)
 *            - sum_{j != k} gamma_jk rho_jk |j><k|.
 *   N          2 .. MLN_MAX_N.
 *   rates      N x N row-major doubles, rates[b * N + a] = gamma_{b->a} >= 0,
 *              1/s (a diagonal entry b = a dephases every coherence of level a
 *              by gamma/2), or NULL for none.
 *   dephasing  N x N row-major doubles, gamma_jk >= 0 in 1/s, symmetric
 *              (gamma_jk == gamma_kj exactly, so that G preserves Hermiticity);
 *              diagonal entries are not read. NULL for none.
 *   G_out      caller-owned (N*N) x (N*N) complex superoperator (2 N^4
 *              doubles, interleaved), on row-major vec(rho); overwritten.
 * The result preserves trace and Hermiticity and is accepted by mln_create.
 * Errors: MLN_EINVAL (N out of range, NULL G_out, a negative or non-finite
 * rate, asymmetric dephasing), message in mln_create_error.
 */
mln_status mln_lindblad_superop(int32_t N, const double *rates, const double *dephasing, double *G_out);

/*
 * Diagnostic: evaluate on the device, for n angles x (host array), the pair
 * (sin x, cos x - 1) exactly as the step kernels of the given precision do,
 * into host arrays s and c1. Synchronous; uses the legacy default stream and
 * allocates temporary device memory.
 */
mln_status mln_rotation_terms(int32_t precision, const double *x, int64_t n, double *s, double *c1);

/*
 * Diagnostic: C = A B^T computed by the tensor-core product path of
 * MLN_KERNEL_TENSOR, with A staged in tensor memory (a_in_tmem != 0, as for
 * the state y) or in shared memory (a_in_tmem == 0, as for dz): A split into
 * TF32 high and low parts on the device, B (given in FP64) split on the host,
 * three tcgen05.mma kind::tf32 per K block, FP32 accumulation. Shapes: M = 128 and (nc, kc) one of (32, 40), (48, 32),
 * (48, 40), (32, 24), (16, 8) (MLN_EINVAL otherwise).
 *   A  host, 128 x kc row-major floats;  B  host, nc x kc row-major doubles;
 *   C  host, 128 x nc row-major floats (out).
 * Synchronous, allocates temporary device memory, legacy default stream.
 * MLN_ETIMEOUT if the completion wait gave up.
 */
mln_status mln_tc_product(int32_t nc, int32_t kc, int32_t a_in_tmem, const float *A, const double *B, float *C);

/*
 * Diagnostic: C = A B^T computed by the product path of MLN_KERNEL_TENSOR in
 * the rotated basis (MLN_FORM_ROTATED): A scaled by a power of two (largest
 * magnitude into (2^12, 2^13]) and split into FP16 high and low parts on the
 * device, staged in tensor memory; each row of B (given in FP64) scaled by its
 * own power of two and split into FP16 parts on the host; three tcgen05.mma
 * kind::f16 per K block of 16 (hi*hi, hi*lo, lo*hi), FP32 accumulation, the
 * scales undone on the result. Shapes: M = 128 and (nc, kc) one of (48, 48),
 * (32, 32), (16, 16) (MLN_EINVAL otherwise).
 *   A  host, 128 x kc row-major floats;  B  host, nc x kc row-major doubles;
 *   C  host, 128 x nc row-major floats (out).
 * Synchronous, allocates temporary device memory, legacy default stream.
 * MLN_ETIMEOUT if the completion wait gave up.
 */
mln_status mln_tc_product_f16(int32_t nc, int32_t kc, const float *A, const double *B, float *C);

/*
 * Failure-detection self-test: runs the product kernel above with its MMA and
 * commit left out, so nothing arrives on the completion mbarrier and the
 * kernel's bounded wait (the same as in MLN_KERNEL_TENSOR steps) runs out; the
 * kernel then releases its tensor memory and returns, and the host reads the
 * flag. Returns MLN_ETIMEOUT when that happened (the expected outcome), MLN_OK
 * if the wait somehow completed, MLN_EUNSUPPORTED without a tcgen05 device.
 * Synchronous; the device stays usable. Not part of the paper's method.
 */
mln_status mln_tc_wait_selftest(void);

/*
 * mln_step_noalloc -- the fused step for callers that cannot allocate device
 * memory. (Not a part of the paper's method: it has no counterpart there.)
 *
 * Who needs it: code that may not call cudaMalloc or any allocating library
 * routine once it runs -- a host application whose device memory is owned by
 * its own pool or framework, a plug-in that must not grow the process's
 * device footprint, a loop with a fixed memory budget. mln_create allocates
 * the context's second copy of the state and fields, its flag word and its
 * conversion tables; this call allocates nothing. It runs the same
 * register-model step kernel (MLN_KERNEL_REGISTER) as mln_step, and keeps the
 * second copy of the state and fields and the flag word in one fixed
 * file-scope device array of MLN_STATIC_SCRATCH_BYTES (32 MiB), which every
 * GPU that loads this library holds until the process exits.
 *
 *   p           problem (as for mln_create; kernel MLN_KERNEL_AUTO or
 *               MLN_KERNEL_REGISTER -- both run the register model here -- form
 *               not MLN_FORM_ROTATED, field solver MLN_MAXWELL_FDTD; otherwise
 *               MLN_EINVAL).
 *   d_state, Ez, Hy  caller-owned device buffers with the sizes and layout of
 *               mln_query_buffers: the state in, the state after n_steps out.
 *   init_state  non-zero: first write the initial medium state built from
 *               rho0 into d_state (Ez, Hy are used as given).
 *   n_steps     steps to queue (>= 0); src as for mln_step (samples 0 ..
 *               n_steps-1 of this call).
 *   stream      cudaStream_t for all work (NULL: legacy default stream).
 *
 * The problem must fit: 256 + align256(state bytes) + 2 * align256(n_cells *
 * real size) <= MLN_STATIC_SCRATCH_BYTES, else MLN_EINVAL with a message
 * (mln_create_error). The FP64 set-up runs on the host at every call (host
 * heap only). The first call on each device looks up the array's device
 * address with that device current (cudaGetSymbolAddress) and keeps it,
 * looking it up again when the device's context has changed (for instance
 * after cudaDeviceReset); make that first call, and the first call after such
 * a change, before any stream capture. Every call shares the one array
 * and leaves its contents behind (the flag word is cleared at each call), so
 * calls whose work overlaps on the GPU -- on different streams, or from
 * different threads -- race and corrupt each other's results: serialise them.
 * Work is queued asynchronously; non-finite values are not reported.
 */
#define MLN_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)
mln_status mln_step_noalloc(const mln_params *p, void *d_state, void *Ez, void *Hy, int32_t init_state,
                            int64_t n_steps, const double *src, void *stream);

/*
 * Diagnostic: the CUDA source that MLN_KERNEL_JIT would compile for p (the
 * merged form; the rotated basis when p->form is MLN_FORM_ROTATED), written to
 * buf (capacity cap bytes, NUL-terminated when it fits);
 * *len receives the length without the NUL. Host only.
 */
mln_status mln_kernel_source(const mln_params *p, char *buf, size_t cap, size_t *len);

/* Library version string. */
const char *mln_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MLN_H */
