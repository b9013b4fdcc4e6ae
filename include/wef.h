/*
 * wef.h - C ABI of the GB300 Wigner-Eckart factorized Boltzmann collision operator.
 *
 * The library evaluates, for a batch of velocity-space cells, the bilinear
 * Galerkin collision operator
 *
 *     Q_{k1,q1} = sum_c sum_{k2,k3} R^{(c)}_{k1 k2 k3} Phi^{(c,q1)}_{k2 k3},
 *     Phi^{(c,q1)}_{k2 k3} = sum_{z in slice (c,q1)} g_z f_{k2,q2z} f_{k3,q3z}
 *
 * (the angular-first contraction of Sec. 4.5.4 of the paper, itself a
 * rearrangement of the full discrete sum of Sec. 4.5 and of the dense form
 * Q_a = sum_bc C_abc f_b f_c of Sec. 2.3 with C = R * G_R, Sec. 4.1).
 *
 * Basis and layout conventions (Sec. 2.2, Sec. 4.1):
 *   K  = Kmax + 1 radial functions R_kl(v) = N_kl v^l L_k^{(l+1/2)}(v^2/2),
 *        orthonormal under M(v) = (2 pi)^{-3/2} exp(-v^2/2) (identity mass matrix);
 *   NQ = (Lmax+1)^2 real spherical harmonics Y_lm (no Condon-Shortley phase,
 *        cos-type for m > 0, sin-type for m < 0), angular index q = l^2 + l + m;
 *   one cell = K * NQ doubles, index k * NQ + q (cells contiguous: [ncells][K][NQ]).
 *   Channels c = (l1,l2,l3) are enumerated l1 outermost, then l2, then l3
 *   ascending, triangle rule, l1+l2+l3 even, all <= Lmax (Sec. 4.6).
 *   The core is R[c][k1][k2][k3] (FP64), c in that order.
 *   The real Gaunt weight of a COO row is g = integral over S^2 of
 *   Y_q1 Y_q2 Y_q3 (Table 1 prints these values).
 *
 * Ownership: the caller owns every pointer it passes; the library copies what
 * it keeps (tables and the uploaded core live on the device until
 * wef_destroy).  Device pointers are plain CUDA device addresses; host
 * pointers are plain host addresses.
 *
 * Errors: every call returns a wef_status; on failure wef_last_error() gives a
 * thread-local message.  No call throws across the ABI.  NaN/Inf in the inputs
 * propagate to the outputs and are not checked.
 */
#ifndef WEF_H
#define WEF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wef_operator* wef_op;

typedef enum {
  WEF_OK = 0,
  WEF_EINVAL = -1,  /* bad argument (null pointer, size out of range, misaligned buffer) */
  WEF_ENOMEM = -2,  /* device or host allocation failed */
  WEF_ECUDA = -3,   /* a CUDA runtime call failed (message has the CUDA error string) */
  WEF_ENOCORE = -4, /* evaluate called before wef_upload_core */
  WEF_ESHAPE = -5,  /* (Kmax, Lmax) outside the supported range or mismatched lengths */
  WEF_ETIMEOUT = -6 /* a bounded device-side wait gave up (status word set by a kernel) */
} wef_status;

typedef enum {
  WEF_FP64 = 0,       /* everything in FP64 (angular coupling and radial contraction) */
  WEF_MIXED_BF16 = 1, /* FP64 angular coupling, BF16 x BF16 -> FP32 radial stage on tcgen05 */
  WEF_MIXED_TF32 = 2, /* FP64 angular coupling, TF32 x TF32 -> FP32 radial stage on tcgen05 */
  WEF_RADIAL_FP32 = 3, /* radial-first ordering: both radial contractions in FP32 on the CUDA cores,
                          Gaunt-weighted angular reduction in FP64 (Sec. 4.5.3 made dense) */
  WEF_RADIAL_TC = 4    /* radial-first ordering as WEF_RADIAL_FP32, the first radial contraction (the
                          core, shared by all cells, times f) on tcgen05 in split TF32 (three TF32
                          products per term, FP32 accumulation); Kmax = 8, 10 or 12.  Taken by the
                          one-shape calls (wef_workspace_size, wef_evaluate and those built on it:
                          wef_evaluate_host, wef_integrate, wef_linearized_apply) and wef_flops; plans
                          and ragged batches refuse it */
} wef_precision;

/* Flags of wef_upload_core. */
#define WEF_CORE_APPLY_NULLSPACE 1u /* zero the Sec. 4.4.2/4.4.3 slices of R before use */

/* Supported sizes: 0 <= Kmax <= 16, 0 <= Lmax <= 20. */
#define WEF_MAX_KMAX 16
#define WEF_MAX_LMAX 20

/*
 * wef_create - build the angular geometry of a (Kmax, Lmax) operator.
 * Sec. 4.1-4.2: channel list, real Gaunt table (exact Wigner 3-j values turned
 * real by the unitary complex->real map), slices (c, q1), and the device
 * programs of the evaluation kernels.  gamma is the cross-section exponent of
 * B = u^gamma / (4 pi) (0 Maxwell molecules, 1 hard spheres, 0.5 VHS); it is
 * only recorded here (the core carries the physics).  Host only: the device
 * copies are made by the first wef_upload_core, on the device current then, and
 * the operator is bound to that device until wef_destroy.
 * Errors: WEF_EINVAL (out NULL, gamma outside [0, 2]), WEF_ESHAPE (Kmax or Lmax
 * out of range), WEF_ENOMEM.
 */
wef_status wef_create(int kmax, int lmax, double gamma, wef_op* out);

/* Sizes of the operator: N = K*NQ per cell (Sec. 2.2: K radial functions times NQ real
 * harmonics), number of channels N_T (Sec. 4.6), Gaunt nonzeros N_G (Sec. 4.2, Table 6),
 * and the core length N_T*K^3 (doubles; Sec. 4.3).  Any out pointer may be NULL.
 * Errors: WEF_EINVAL (op NULL). */
wef_status wef_sizes(wef_op op, int64_t* n_per_cell, int64_t* n_channels, int64_t* n_gaunt, int64_t* core_len);

/* Copy the COO table of Table 1 order (q3 slowest, q1 fastest; 0-based
 * indices) into host arrays of length >= N_G.  Any array may be NULL.
 * Errors: WEF_EINVAL (op NULL). */
wef_status wef_gaunt_coo(wef_op op, int32_t* q1, int32_t* q2, int32_t* q3, int32_t* c, double* g);

/*
 * wef_upload_core - copy a core R[c][k1][k2][k3] (FP64 host array of length
 * N_T*K^3) to the device and derive the per-precision operand tables.  With
 * WEF_CORE_APPLY_NULLSPACE, the mass/momentum/energy slices (Sec. 4.4.2) and the
 * detailed-balance slice R^{(000)}_{k1,0,0} (Sec. 4.4.3) are zeroed first.
 * Synchronous.  The caller keeps R_host.  May be called again to replace the core.
 * The first call binds the operator to the current device; later calls (and every
 * evaluation) must be made with that device current.
 * Errors: WEF_EINVAL (NULL argument, another device current), WEF_ESHAPE (len),
 * WEF_ECUDA (device allocation or copy; the previous core is then released).
 */
wef_status wef_upload_core(wef_op op, const double* R_host, int64_t len, unsigned flags);

/* Bytes of device workspace wef_evaluate needs for ncells cells (256-byte aligned use).
 * Errors: WEF_EINVAL (op or bytes NULL, ncells < 0, unknown precision). */
wef_status wef_workspace_size(wef_op op, int64_t ncells, wef_precision prec, int64_t* bytes);

/*
 * wef_evaluate - Q = Q(f, f) for ncells cells on `stream` (asynchronous).
 * f_dev, q_dev: device arrays [ncells][K][NQ] FP64 (may not alias).
 * workspace: device buffer of at least wef_workspace_size bytes, 256-byte aligned;
 * it is scratch (overwritten), and calls that share it must be ordered on the GPU.
 * stream: a cudaStream_t (NULL = legacy default stream).  Allocates nothing.
 * The conservation projection (Sec. 4.4) writes exact zeros to the mass,
 * momentum and energy outputs (k=0,l=0), (k=0,l=1), (k=1,l=0) of every cell.
 * ncells == 0 is a no-op.
 * Errors (checked before anything is queued): WEF_EINVAL (op or a buffer NULL, unknown
 * precision, ncells < 0 or above 65535 * 32 * 1024, workspace unaligned or too small, a device other
 * than the operator's current), WEF_ENOCORE (no core uploaded); WEF_ECUDA if a launch
 * fails.
 */
wef_status wef_evaluate(wef_op op, const double* f_dev, double* q_dev, int64_t ncells, wef_precision prec,
                        void* workspace, int64_t workspace_bytes, void* stream);

/*
 * Ragged batches (several (Kmax, Lmax) operators in one launch).
 *
 * A plan covers the cells of nops operators stored back to back in one buffer:
 * first ncells[0] cells of ops[0] (each K0*NQ0 doubles, layout as above), then
 * ncells[1] cells of ops[1], and so on; Q uses the same layout.  It evaluates them
 * with one re-tiling launch and one persistent tensor-core launch (one CTA per SM
 * pulling (shape, tile, task range) work items from a device queue, longest
 * first).  granularity = how many task ranges each 32-cell tile is split into
 * (0 = from the tuning cache named by the WEF_TUNE_CACHE environment variable,
 * else about 8 items per SM).  Precision: WEF_MIXED_TF32 or WEF_MIXED_BF16.
 * With WEF_RADIAL_FP32 the plan runs the radial-first evaluation of each shape (one
 * persistent launch per shape, largest first) on `granularity` concurrent forked
 * streams (0 = cache, else 4), joined back to the caller's stream; its autotuned setting
 * also fixes the launches' L2 tile-group size.
 * Every operator must have a core uploaded (Kmax >= 1 for the tensor-core path) and
 * must outlive the plan.
 * Set-up allocations happen in wef_plan_create only.
 * Errors: wef_plan_create - WEF_EINVAL (NULL argument, nops < 1, negative count, a
 * precision other than those above), WEF_ENOCORE, WEF_ESHAPE (Kmax = 0 on the
 * tensor-core path), WEF_ECUDA / WEF_ENOMEM (set-up); the launching calls - WEF_EINVAL
 * (NULL plan or buffer, workspace unaligned or smaller than wef_plan_workspace_size),
 * the errors of wef_evaluate for a shape's evaluation, WEF_ECUDA (launch, capture).  On
 * an error the forked streams are still joined back to `stream`.
 */
typedef struct wef_plan_s* wef_plan;
wef_status wef_plan_create(const wef_op* ops, const int64_t* ncells, int nops, wef_precision prec, int granularity,
                           wef_plan* out);
/* Bytes of device workspace (256-byte aligned) the plan's launches need. */
wef_status wef_plan_workspace_size(wef_plan plan, int64_t* bytes);
/* Asynchronous evaluation on `stream`; allocates nothing. */
wef_status wef_plan_execute(wef_plan plan, const double* f_dev, double* q_dev, void* workspace, int64_t ws_bytes,
                            void* stream);
/* Same, replayed from a CUDA graph: the first call (and any call with different
 * buffers) captures the launches on the plan's own stream and instantiates the
 * graph; later calls only launch it on `stream`. */
wef_status wef_plan_graph_launch(wef_plan plan, const double* f_dev, double* q_dev, void* workspace,
                                 int64_t ws_bytes, void* stream);
/* Autotuner: times the plan at granularities 1, 2, 4, ... (radial-first: 1, 2, 4, 8
 * streams, each with L2 tile groups of 12, 24 and 48 MB of FP32 tiles - the group bounds
 * what a group's tiles and Q rows occupy in L2) on the given buffers (synchronous), keeps
 * the fastest, appends it to the WEF_TUNE_CACHE file if set, and returns it in *chosen
 * (may be NULL; radial-first: streams + 16 * group MB). */
wef_status wef_plan_autotune(wef_plan plan, const double* f_dev, double* q_dev, void* workspace, int64_t ws_bytes,
                             void* stream, int* chosen);
/* Synchronous check of the plan's device status word (see wef_device_status). */
wef_status wef_plan_status(wef_plan plan, int reset);
wef_status wef_plan_destroy(wef_plan plan);

/*
 * wef_evaluate_ragged - Q = Q(f, f) for a batch mixing cells of several operators, each cell
 * anywhere in f and q: the bilinear form of Sec. 2.3, Q_a = sum_bc C_abc f_b f_c, evaluated
 * per cell by the contraction of Sec. 4.5 that `prec` selects (WEF_RADIAL_FP32: the Sec.
 * 4.5.3 ordering with FP32 radial stages and an FP64 Gaunt reduction; WEF_FP64: the
 * Sec. 4.5.4 angular-first contraction in FP64), with the Sec. 4.4 projection.
 *   ops[0..nops-1]: 1 <= nops <= WEF_RAGGED_MAX_OPS operators with uploaded cores, all on the
 *     current device (host array of handles; the operators must outlive the queued work).
 *   shape_id_dev[i] (device, int32, ncells entries): the operator of cell i, an index into
 *     ops; cells with an index outside [0, nops) are skipped (their Q is not written).
 *   offset_dev[i] (device, int64): where cell i's K*NQ values start, in doubles from f_dev;
 *     its Q is written at the same offset from q_dev (layout k*NQ + q of its operator).
 *     Cells must not overlap in q_dev; f and q may not alias.
 *   workspace: device, 256-byte aligned, at least wef_ragged_workspace_size bytes (which
 *     depends only on the operators, ncells and prec); scratch, overwritten.
 * Asynchronous on `stream`, allocates no device memory, reads nothing back to the host: the
 * batch's composition is worked out on the device (per-operator counts, cell lists and
 * 32-cell tiles, set up by kernels on `stream`), then each operator's contraction runs over
 * its own tiles on one of a few streams forked from `stream` and joined back to it.  Each
 * cell's result is bitwise the one wef_evaluate gives for that cell at the same precision.
 * The forked streams belong to the caller's stream and are created by the first call with
 * that stream on a device (make that call before any stream capture); calls on different
 * streams overlap; calls from several host threads take turns queueing their work.
 * Errors (checked before anything is queued): WEF_EINVAL (NULL argument, nops out of range,
 * a precision other than the two above, ncells < 0 or too large, workspace unaligned or too
 * small, an operator on another device), WEF_ENOCORE; WEF_ECUDA if a launch fails.
 * ncells == 0 is a no-op.
 */
#define WEF_RAGGED_MAX_OPS 32
wef_status wef_ragged_workspace_size(const wef_op* ops, int nops, int64_t ncells, wef_precision prec, int64_t* bytes);
wef_status wef_evaluate_ragged(const wef_op* ops, int nops, const int32_t* shape_id_dev, const int64_t* offset_dev,
                               const double* f_dev, double* q_dev, int64_t ncells, wef_precision prec,
                               void* workspace, int64_t ws_bytes, void* stream);

/*
 * Evaluation from host memory: the same Q(f, f) for f and Q in host memory (pinned for
 * the copies to be asynchronous), streamed through the device in chunks of chunk_cells
 * cells so that the host<->device copies of one chunk overlap the evaluation of another.
 * The workspace (wef_host_workspace_size(op, chunk_cells, prec), 256-byte aligned, device
 * memory) holds one chunk's evaluation workspace and two staging slots each for f and Q.
 * Copies run on two library streams ordered by events; evaluations run on `stream`, which
 * also waits for the last copy back: q_host is complete once `stream` has.  Calls on one
 * operator must not overlap.  Errors as wef_evaluate.
 */
wef_status wef_host_workspace_size(wef_op op, int64_t chunk_cells, wef_precision prec, int64_t* bytes);
wef_status wef_evaluate_host(wef_op op, const double* f_host, double* q_host, int64_t ncells, int64_t chunk_cells,
                             wef_precision prec, void* workspace, int64_t ws_bytes, void* stream);

/*
 * Unfactorised baselines (Sec. 4.5): the same Q(f, f), FP64, without the factorisation,
 * for comparison on the same GPU.  Both use the uploaded (symmetrised, zeroed) core.
 *
 * wef_naive_evaluate: the COO loop of Sec. 4.5.2 - for every non-zero Gaunt entry the
 *   full K^3 radial sum.  f_dev, q_dev: [ncells][K][NQ]; workspace: at least
 *   wef_workspace_size(op, ncells, WEF_FP64) bytes, 256-byte aligned.  Asynchronous.
 * wef_dense_tensor_size / wef_dense_assemble: the dense tensor C[a1][a2][a3] of Sec. 4.5.1
 *   (N^3 doubles, N = K NQ; 85 GB at Kmax = Lmax = 12) written by the library into a
 *   caller-owned device buffer; rows of the collision invariants are zero.
 * wef_dense_evaluate: Q_a1 = sum_{a2,a3} C[a1][a2][a3] f_a2 f_a3 as two cuBLAS FP64 GEMMs
 *   per chunk of cells (chunk = ws_bytes / (N^2 * 8); wef_dense_workspace_size suggests
 *   a workspace for up to 256 cells per chunk).  Asynchronous on `stream`.
 * Errors: WEF_EINVAL (NULL buffer, short buffer or workspace), WEF_ENOCORE, WEF_ECUDA.
 */
wef_status wef_naive_evaluate(wef_op op, const double* f_dev, double* q_dev, int64_t ncells, void* workspace,
                              int64_t ws_bytes, void* stream);
wef_status wef_dense_tensor_size(wef_op op, int64_t* bytes);
wef_status wef_dense_assemble(wef_op op, double* C_dev, int64_t bytes, void* stream);
wef_status wef_dense_workspace_size(wef_op op, int64_t ncells, int64_t* bytes);
wef_status wef_dense_evaluate(wef_op op, const double* C_dev, const double* f_dev, double* q_dev, int64_t ncells,
                              void* workspace, int64_t ws_bytes, void* stream);

/*
 * Time integration and linearization (device).
 *
 * wef_integrate advances the spatially homogeneous equation df/dt = Q(f, f)
 * (Sec. 2.1) in place by nsteps classical fourth-order Runge-Kutta steps of size
 * dt (the explicit time stepping of Sec. 5.3.2), every cell independently, with Q
 * evaluated at precision `prec`.  Because the projection zeroes the mass, momentum
 * and energy components of every Q exactly, those components of f do not change.
 * wef_linearized_apply computes out = L d, L = dQ/dc at the base states c0
 * (Sec. 5.3.1), as Q(c0 + d) - Q(c0) - Q(d) (exact for the bilinear form; relative
 * rounding grows like |c0| / |d|).  Both are asynchronous on `stream`, allocate
 * nothing, and need a workspace of wef_integrate_workspace_size bytes (256-byte
 * aligned).  c0, d, out: [ncells][K][NQ]; out may not alias the inputs.
 */
wef_status wef_integrate_workspace_size(wef_op op, int64_t ncells, wef_precision prec, int64_t* bytes);
wef_status wef_integrate(wef_op op, double* f_dev, int64_t ncells, double dt, int nsteps, wef_precision prec,
                         void* workspace, int64_t ws_bytes, void* stream);
wef_status wef_linearized_apply(wef_op op, const double* c0_dev, const double* d_dev, double* out_dev, int64_t ncells,
                                wef_precision prec, void* workspace, int64_t ws_bytes, void* stream);

/*
 * Devices: an operator lives on the device that was current when its core was first
 * uploaded; evaluation calls must be made with that device current (WEF_EINVAL otherwise).
 */

/*
 * wef_core_build - the kinematic core R[c][k1][k2][k3] of the operator by the
 * singular quadrature of Sec. 4.3 / Appendix A-B, on the host (all cores of the
 * machine).  pad_rad / pad_ang are the selective paddings of Appendix B (the
 * paper uses 10-20).  R_out: host array of length N_T*K^3.  Raw core: no
 * conservation zeroing is applied (pass WEF_CORE_APPLY_NULLSPACE to upload).
 * Errors: WEF_EINVAL (NULL argument, padding outside [0, 200]), WEF_ESHAPE (len).
 */
wef_status wef_core_build(wef_op op, int pad_rad, int pad_ang, double* R_out, int64_t len);

/*
 * wef_core_build_device - the same core by the same quadrature (Sec. 4.3, Appendix A-B:
 * rules, point counts, paddings, Funk-Hecke sphere means) assembled on the current GPU
 * in FP64: point tables per chunk of z nodes, then one CTA per channel accumulating the
 * rank-1 radial terms.  Synchronous; allocates its device scratch (about 1 GB at most
 * for the point tables plus the core) and frees it before returning.  R_out: host array
 * of length N_T*K^3, the raw core as wef_core_build returns it (agrees with it to
 * rounding).  Errors: WEF_EINVAL, WEF_ESHAPE (len), WEF_ECUDA.
 */
wef_status wef_core_build_device(wef_op op, int pad_rad, int pad_ang, double* R_out, int64_t len);

/*
 * wef_flops - arithmetic the evaluation executes per cell: FP64 flops (angular
 * coupling, plus the radial contraction for WEF_FP64) and tensor-core flops
 * (radial contraction, padded MMA shapes, for the mixed precisions).  An FMA
 * counts as 2.  For WEF_RADIAL_FP32 the second output is the FP32 CUDA-core work of
 * the two radial contractions instead; for WEF_RADIAL_TC the tensor-core work of the
 * first radial contraction as executed (three TF32 products per term on tiles padded to
 * 16 k2 x 16 K columns, the 32 cells of a tile repeated over the four tensor-memory lane
 * quadrants).  Derived from the operator's programs; any
 * out pointer may be NULL.  Errors: WEF_EINVAL (op NULL, unknown precision).
 */
wef_status wef_flops(wef_op op, wef_precision prec, double* fp64_flops_per_cell, double* tc_flops_per_cell);

/*
 * wef_set_trace_events - tracing hook: when ev_start/ev_stop (cudaEvent_t) are
 * non-NULL, the next wef_evaluate calls record ev_start on the stream just before
 * the dominant (contraction) kernel and ev_stop just after it, so callers can
 * time that kernel alone.  Pass NULLs to switch tracing off.  The events stay the
 * caller's and must outlive the calls that record them.  Errors: WEF_EINVAL (op NULL).
 */
wef_status wef_set_trace_events(wef_op op, void* ev_start, void* ev_stop);

/*
 * wef_device_status - synchronous check of the operator's device status word:
 * WEF_ETIMEOUT if any earlier evaluation had a bounded in-kernel wait (mbarrier
 * on a tensor-core or bulk-copy completion) give up, in which case that
 * evaluation's outputs are incomplete; WEF_OK otherwise.  reset != 0 clears the
 * word.  The word is shared by all evaluations of the operator.
 */
wef_status wef_device_status(wef_op op, int reset);

/*
 * wef_evaluate_noalloc - the FP64 evaluation of wef_evaluate (prec = WEF_FP64)
 * for callers that cannot allocate device memory when they evaluate: it takes no
 * workspace and allocates nothing, using instead a fixed scratch array of
 * WEF_NOALLOC_SCRATCH_BYTES that the library keeps in device memory on every GPU
 * that loads it, until the process exits.  The paper has no counterpart; this is
 * a deployment convenience.
 *   - Size limit: ncells * K * NQ * 8 bytes, rounded up to whole 32-cell tiles,
 *     must fit the scratch (928 cells at Kmax = Lmax = 12); larger batches are
 *     rejected with WEF_EINVAL and a message giving the limit.
 *   - The first call on each device looks up the scratch's device address (with
 *     that device current), which is also when CUDA loads the library module holding
 *     the array, making its 16 MiB resident with an implicit device synchronisation;
 *     make that first call at set-up, before any stream capture.  Later calls
 *     allocate nothing.
 *   - All calls on a device share the one scratch array, which keeps the last
 *     call's contents: calls that overlap on the GPU (other streams, other
 *     threads) race and must be ordered by the caller.
 *   - Same arguments, results and errors as wef_evaluate otherwise.
 */
#define WEF_NOALLOC_SCRATCH_BYTES (16u << 20)
wef_status wef_evaluate_noalloc(wef_op op, const double* f_dev, double* q_dev, int64_t ncells, void* stream);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* wef_last_error(void);

/* Release the operator and its device memory.  NULL is accepted. */
wef_status wef_destroy(wef_op op);

#ifdef __cplusplus
}
#endif

#endif /* WEF_H */
