/*
 * tfmm - Tucker-compressed FMM far-fields on one GPU (C ABI).
 *
 * The library implements the setup and the two per-iteration stages of
 * "Compression of Far-Fields in the Fast Multipole Method via Tucker
 * Decomposition" (Qian, Wang, Yucel, arXiv 2103.05822):
 *
 *   setup    RWG functions on a triangle mesh (Sec. II.A, ref. [20]); the
 *            FMM-FFT box grid (Sec. II.A); the (L+1) x N_phi spherical grid
 *            (Sec. II.A after Eq. 4); far-field tensors of every group (Eq. 4,
 *            Fig. 1a); truncated HOSVD (Eq. 6, Sec. II.B).
 *   hot path aggregation from the Tucker factors (Fig. 2b, replacing Eq. 3)
 *            and disaggregation (Fig. 3b, replacing Eq. 5), plus the same two
 *            stages from the uncompressed tensors (Eqs. 3 and 5) for comparison.
 *
 * Conventions used by every entry point:
 *   - Complex numbers are interleaved pairs (re, im): tfmm_cfloat (8 bytes) on
 *     the hot path, tfmm_cdouble (16 bytes) for setup inputs and exports.
 *   - A "direction" index is i = i_theta + n_theta * i_phi (theta fastest).
 *   - Right-hand-side blocks are column-major: x[n + ldx * r] is RWG n of RHS r.
 *   - Spectra are laid out [R][G][2][n_phi][n_theta]: RHS r, group g, component
 *     alpha (0 = theta, 1 = phi), direction i at
 *     ((r * G + g) * 2 + alpha) * N_dir + i.  Groups are the non-empty boxes in
 *     ascending linear box index ix + Kx (iy + Ky iz).
 *   - Pointers documented "device" must be CUDA device (or managed) memory on
 *     the current device; "host" pointers are ordinary CPU memory.  The caller
 *     owns every buffer it passes; the library copies what it keeps.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Hot-path calls are asynchronous on that stream; calls on one
 *     plan must be ordered on one stream (a plan's work queue is shared).
 *   - Every function returns a tfmm_status and never aborts the process.
 *     tfmm_last_error() returns a message for the last failure of the calling
 *     thread.  Asynchronous kernel faults surface at the next call that
 *     synchronises.
 */
#ifndef TFMM_H
#define TFMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TFMM_OK = 0,
    TFMM_INVALID_ARG = 1, /* bad pointer, size, layout or parameter */
    TFMM_OOM = 2,         /* device or host allocation failed */
    TFMM_CUDA = 3,        /* CUDA runtime / cuBLAS / cuSOLVER error */
    TFMM_NUMERIC = 4,     /* eigen-solver failure or non-finite data */
    TFMM_NOT_BUILT = 5,   /* the requested data was not built (e.g. dense tensors) */
    TFMM_IO = 6           /* checkpoint file could not be read or written */
} tfmm_status;

typedef struct { float re, im; } tfmm_cfloat;
typedef struct { double re, im; } tfmm_cdouble;

typedef struct tfmm_mesh tfmm_mesh;
typedef struct tfmm_plan tfmm_plan;

/* Setup parameters (Sec. II.A and III).  Fill with tfmm_params_default(). */
typedef struct {
    double k;          /* wavenumber 2 pi / lambda (> 0) */
    double box;        /* FMM box edge a (> 0), same length unit as the mesh */
    double digits;     /* FMM accuracy d0 in digits (> 0), sets L (Sec. II.A) */
    int32_t nphi_rule; /* 0: N_phi = 2L+1 (the paper), 1: N_phi = 2(L+1) */
    int32_t L_override;/* > 0: use this L instead of the bandwidth formula */
    double tol;        /* Tucker tolerance gamma (>= 0), truncation gamma/sqrt(3) per mode */
    int32_t quad_order;/* collapsed Gauss-Legendre order per triangle, 1..10 (default 5) */
    int32_t keep_dense;/* nonzero: also keep FP32 uncompressed tensors (Eqs. 3, 5) */
    int32_t max_rhs;   /* largest R later passed to the hot path (>= 1) */
    int32_t batch_groups; /* groups per setup batch (0 = automatic) */
    int32_t mrhs_precision; /* engine for R > 1: 0 = grouped-GEMM chain in FP32 on CUDA cores;
                               1 = the single-RHS kernels, one column after another (FP32);
                               2 or 3 = tensor cores with FP32 operands split into 2 or 3
                               BF16 terms (hi + lo [+ lo2]), FP32 accumulation */
    int32_t compression; /* 0 = Tucker (Eq. 6, gamma / sqrt(3) per mode); 1 = truncated SVD of
                            the N_dir x n_beta aggregation matrix at gamma, the comparator of
                            Sec. II.C and Tables I-IV, stored as a Tucker format with identity
                            theta / phi factors (r_theta = n_theta, r_phi = n_phi), core
                            (U_r Sigma_r)^T and U_beta = conj(V_r); its hot path skips the
                            theta / phi steps and runs the single-RHS kernels for every R */
    int32_t reserved[4];
} tfmm_params;

typedef struct {
    int32_t L, n_theta, n_phi, n_dir;
    int32_t n_groups;
    int32_t K[3];             /* box grid K_x, K_y, K_z */
    int64_t n_rwg;
    int32_t max_n_beta;
    int32_t max_rank[3];      /* largest r_theta, r_phi, r_beta over groups and alpha */
    int64_t tucker_bytes;     /* FP32 factors + cores as stored (with padding) */
    int64_t tucker_bytes_alg; /* FP32 factors + cores without padding */
    int64_t dense_bytes;      /* FP32 uncompressed tensors (0 if not kept) */
    double setup_ms[4];       /* far-field, HOSVD, packing, total */
    int32_t kernel_errors;    /* tensor-core kernels that gave up waiting (0 when healthy) */
    int32_t pad_;
} tfmm_plan_info;

/* Default parameters: k = 2 pi, box 0.5, 3 digits, N_phi = 2(L+1), gamma 1e-4,
 * quadrature order 5, no dense copy, max_rhs 1. */
tfmm_status tfmm_params_default(tfmm_params* p);

/* Message of the last failure on this thread ("" if none).  Valid until the
 * thread's next tfmm call. */
const char* tfmm_last_error(void);

/* ------------------------------------------------------------------ mesh -- */
/* Builds the RWG functions of a triangle mesh (Sec. II.A, ref. [20]).
 * verts: host, nv x 3 doubles (row-major).  tris: host, nt x 3 vertex ids.
 * Every edge shared by exactly two triangles carries one RWG; RWGs are
 * numbered by (min vertex id, max vertex id) of their edge, ascending; T+ is
 * the adjacent triangle with the lower index.  The arrays are copied.
 * Errors: INVALID_ARG for null pointers, nv < 3, nt < 1, out-of-range or
 * repeated vertex ids in a triangle, degenerate (zero-area) triangles. */
tfmm_status tfmm_mesh_create(const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                             tfmm_mesh** out);
tfmm_status tfmm_mesh_num_rwg(const tfmm_mesh* mesh, int64_t* n_rwg);
/* Host outputs, each n_rwg x 2 (row-major): edge vertex ids, (T+, T-) triangle
 * ids, free vertex ids (p+, p-).  Any output may be NULL. */
tfmm_status tfmm_mesh_rwg(const tfmm_mesh* mesh, int64_t* edge, int64_t* tri, int64_t* free_vertex);
tfmm_status tfmm_mesh_destroy(tfmm_mesh* mesh);

/* ------------------------------------------------------------------ plan -- */
/* Runs the whole setup on the current GPU: box grid and groups (Sec. II.A),
 * bandwidth L and grid, far-field tensors by Eq. 4 in FP64, truncated
 * sequential HOSVD (Eq. 6) in FP64, FP32 packing of factors and cores for the
 * hot path, and (keep_dense) the FP32 uncompressed tensors.  `stream` orders
 * the setup work; the call returns after the setup has finished.
 * Errors: INVALID_ARG (parameters), OOM, CUDA, NUMERIC. */
tfmm_status tfmm_plan_create(const tfmm_mesh* mesh, const tfmm_params* p, void* stream, tfmm_plan** out);

/* Builds a plan from Tucker factors given by the caller instead of running the
 * setup (Eq. 6 data, e.g. from another compressor or a checkpoint).
 *   n_rwg         total RWG count (x / y length)
 *   n_groups      G; n_theta, n_phi: grid sizes (N_dir = n_theta n_phi)
 *   group_offsets host, G+1 ascending offsets into group_rwg
 *   group_rwg     host, global RWG ids of each group; every id in 0..n_rwg-1
 *                 appears exactly once over all groups
 *   ranks         host, G x 2 x 3: (r_theta, r_phi, r_beta) per group and alpha
 *   factors       host, FP64 complex, for g = 0..G-1, alpha = 0, 1 in turn:
 *                 U_theta (n_theta x r_theta), U_phi (n_phi x r_phi),
 *                 U_beta (n_beta x r_beta), core (r_theta x r_phi x r_beta),
 *                 each column-major and packed back to back
 *   weights       host, N_dir quadrature weights (NULL: all ones)
 *   max_rhs       largest R the hot path will be called with
 * Errors: INVALID_ARG for inconsistent sizes or ranks outside
 * 1 <= r <= n, OOM, CUDA. */
tfmm_status tfmm_plan_from_tucker(int64_t n_rwg, int32_t n_groups, int32_t n_theta, int32_t n_phi,
                                  const int64_t* group_offsets, const int64_t* group_rwg,
                                  const int32_t* ranks, const tfmm_cdouble* factors,
                                  const double* weights, int32_t max_rhs, void* stream,
                                  tfmm_plan** out);

/* Adds uncompressed tensors to a plan (for the dense stages of Eqs. 3 and 5).
 * tensors: host, FP64 complex, for g, alpha in turn an n_theta x n_phi x n_beta
 * column-major tensor A[i_theta, i_phi, n] = P^{alpha,+}_{n,i} (Fig. 1a). */
tfmm_status tfmm_plan_set_dense(tfmm_plan* plan, const tfmm_cdouble* tensors, void* stream);

/* Engine of the R > 1 hot path (see tfmm_params.mrhs_precision): 0, 1, 2 or 3.
 * When the largest work item does not fit the single-RHS kernels (shared
 * memory), every R, R = 1 included, runs the FP32 grouped-GEMM chain.
 * Tensor-core modes build BF16 planes of the factors on first use (device
 * memory: 2 layouts x 2 or 3 terms of every factor).  INVALID_ARG otherwise. */
tfmm_status tfmm_plan_set_mrhs_precision(tfmm_plan* plan, int32_t precision);

/* Plan sizes and setup times; also synchronises the device to read
 * kernel_errors. */
tfmm_status tfmm_plan_info_get(const tfmm_plan* plan, tfmm_plan_info* info);
/* n_beta and ranks (r_theta, r_phi, r_beta) of group g, component alpha. */
tfmm_status tfmm_plan_group(const tfmm_plan* plan, int32_t g, int32_t alpha, int64_t* n_beta,
                            int32_t* ranks3);
/* Host outputs: offsets (G+1) and global RWG ids (n_rwg) of the groups. */
tfmm_status tfmm_plan_members(const tfmm_plan* plan, int64_t* offsets, int64_t* rwg_ids);
/* Host output: box centres r_v, G x 3 (row-major); NULL-safe no-op for plans
 * built from factors (INVALID_ARG). */
tfmm_status tfmm_plan_centres(const tfmm_plan* plan, double* centres);
/* Host outputs: theta (n_theta), w_theta (n_theta, Gauss-Legendre in cos
 * theta), phi (n_phi); *w_phi = 2 pi / n_phi.  Any may be NULL. */
tfmm_status tfmm_plan_quadrature(const tfmm_plan* plan, double* theta, double* w_theta, double* phi,
                                 double* w_phi);
/* Copies the FP64 factors of (g, alpha) to host buffers sized by
 * tfmm_plan_group (column-major, as in tfmm_plan_from_tucker). */
tfmm_status tfmm_plan_export_factors(const tfmm_plan* plan, int32_t g, int32_t alpha, tfmm_cdouble* U_theta,
                                     tfmm_cdouble* U_phi, tfmm_cdouble* U_beta, tfmm_cdouble* core);
/* Recomputes the FP64 far-field tensors of group g (Eq. 4) on the GPU and
 * copies them to host: A_theta and A_phi, each n_theta x n_phi x n_beta
 * column-major.  Needs a plan made by tfmm_plan_create. */
tfmm_status tfmm_plan_farfield(const tfmm_plan* plan, int32_t g, tfmm_cdouble* A_theta, tfmm_cdouble* A_phi,
                               void* stream);
tfmm_status tfmm_plan_destroy(tfmm_plan* plan);

/* -------------------------------------------------------------- hot path -- */
/* Aggregation (Eq. 3 evaluated as in Fig. 2b): for every group g and alpha,
 * spectra[r][g][alpha] = U_theta (U_phi (C x_3 (U_beta^T x_g))^T)^T, the
 * N_dir far-field of the group's currents.
 *   x       device, n_rwg x R column-major FP32 complex, leading dimension ldx >= n_rwg
 *   R       1 <= R <= max_rhs
 *   spectra device, R x G x 2 x N_dir FP32 complex, overwritten
 * R > 1 runs the engine that tfmm_params.mrhs_precision selects; the first call
 * with a given R and engine allocates its scratch and tile lists (device memory
 * owned by the plan), later calls allocate nothing.
 * Errors: INVALID_ARG (null pointers, R out of range, ldx < n_rwg), OOM, CUDA. */
tfmm_status tfmm_aggregate(tfmm_plan* plan, const tfmm_cfloat* x, int32_t R, int64_t ldx, tfmm_cfloat* spectra,
                           void* stream);

/* Disaggregation (Eq. 5 evaluated as in Fig. 3b), the weighted adjoint of
 * tfmm_aggregate:  y = beta y + sum_alpha A_alpha^H (W .* g_alpha)  with W the
 * quadrature weights (apply_weights != 0) or ones (apply_weights == 0, the
 * plain conjugate transpose of Eq. 5).
 *   spectra device, as produced by tfmm_aggregate
 *   y       device, n_rwg x R column-major, leading dimension ldy >= n_rwg
 *   beta    scale of the old y; beta = 0 overwrites y (old NaNs are dropped)
 * Errors: INVALID_ARG, CUDA. */
tfmm_status tfmm_disaggregate(tfmm_plan* plan, const tfmm_cfloat* spectra, int32_t R, int32_t apply_weights,
                              tfmm_cfloat beta, tfmm_cfloat* y, int64_t ldy, void* stream);

/* The same two stages from the uncompressed FP32 tensors (Eqs. 3 and 5).
 * Errors as above, plus NOT_BUILT when the plan holds no dense tensors. */
tfmm_status tfmm_aggregate_dense(tfmm_plan* plan, const tfmm_cfloat* x, int32_t R, int64_t ldx,
                                 tfmm_cfloat* spectra, void* stream);
tfmm_status tfmm_disaggregate_dense(tfmm_plan* plan, const tfmm_cfloat* spectra, int32_t R, int32_t apply_weights,
                                    tfmm_cfloat beta, tfmm_cfloat* y, int64_t ldy, void* stream);

/* Aggregation followed by disaggregation of the spectra it produced, from and
 * to HOST buffers: copies x (host, n_rwg x R column-major, ld n_rwg) to the
 * device, aggregates, disaggregates with weights and beta = 0, copies y back
 * to host (n_rwg x R) and synchronises `stream`.  The translation stage
 * between them is not part of this library: the outgoing spectra are used as
 * incoming spectra.  dense != 0 uses the uncompressed tensors.  Device
 * buffers are owned by the plan and allocated on the first call for a given R.
 * Errors: INVALID_ARG, NOT_BUILT, OOM, CUDA. */
tfmm_status tfmm_matvec_host(tfmm_plan* plan, const tfmm_cfloat* x_host, tfmm_cfloat* y_host, int32_t R,
                             int32_t dense, void* stream);

/* Translation stage of the FMM-FFT (Sec. II.A, between Eqs. 3 and 5; refs. [7, 8];
 * addition theorem of ref. [25]): the incoming spectra of every group from the
 * outgoing spectra of aggregation,
 *   spectra_in[r][v][alpha](k_i) = (-j k / (16 pi^2)) sum over groups v' far from v of
 *                                  T_L(k_i, r_v - r_v') spectra_out[r][v'][alpha](k_i),
 *   T_L(k, X) = sum_{l=0}^{L} (-j)^l (2l + 1) h_l^(2)(k|X|) P_l(k . X / |X|),
 * where two groups are far when their box indices differ by 2 or more in some
 * coordinate (touching boxes are the near field, not computed here).  Then
 * tfmm_disaggregate(spectra_in, apply_weights = 1) gives the far part of Z x of the
 * EFIE (Eq. 2) for the x that tfmm_aggregate received.  Evaluated as a 3-D FFT
 * convolution over the zero-padded box grid, FP32 (the translation kernel's
 * transform is computed once in FP64).  The first call builds it (device memory
 * owned by the plan: the kernel's transform, N_grid x N_dir complex, and a work
 * grid of N_grid x 2 N_dir complex, N_grid >= (2K_x - 1)(2K_y - 1)(2K_z - 1));
 * later calls allocate nothing.
 *   spectra_out  device, R x G x 2 x N_dir FP32 complex (as tfmm_aggregate writes it)
 *   spectra_in   device, same shape, overwritten; must not alias spectra_out
 * Errors: INVALID_ARG (a plan built from factors has no box geometry), OOM, CUDA. */
tfmm_status tfmm_translate(tfmm_plan* plan, const tfmm_cfloat* spectra_out, int32_t R, tfmm_cfloat* spectra_in,
                           void* stream);

/* RWG-tested plane-wave excitations (Eq. 2): V[m + n_rwg r] =
 * -int b_m(r') . pol_r exp(-j k khat_r . r') dr' for R incidences.
 *   khat, pol  host, R x 3 (row-major) propagation directions and polarisations
 *   V          device, n_rwg x R FP32 complex
 * Errors: INVALID_ARG, CUDA.  Needs a plan made by tfmm_plan_create. */
tfmm_status tfmm_planewave(const tfmm_plan* plan, const double* khat, const double* pol, int32_t R,
                           tfmm_cfloat* V, void* stream);

/* Allocation-free variant of tfmm_planewave.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory while they
 * call the library, such as applications whose device memory is all handed out
 * by their own pool allocator (a cudaMalloc from the library would fail or
 * fragment that pool) or loops that cannot afford the device-wide
 * synchronisation a cudaFree implies.  Instead of a per-call allocation, the
 * incidence table is staged in one fixed array inside the library: at most
 * 1024 incidences (48 KiB), present on every GPU that loads the library until
 * the process exits.  The call allocates and frees no memory.  khat and pol are
 * first copied into a fixed host array of the library (ordinary pageable
 * memory) and from there to the device table, so the caller may reuse or free
 * its arrays, pinned or not, as soon as the call returns; a copy from pageable
 * memory may make the call wait for work queued earlier on `stream`.  The
 * kernel itself is queued on `stream` without waiting for it.
 *   khat, pol  host, R x 3, as tfmm_planewave
 *   V          device, n_rwg x R FP32 complex, overwritten
 *   R          1..1024; a larger R returns INVALID_ARG with a message
 * The first call on a device looks up the device address of the table (once
 * per device, with that device current).  Every call shares the one table and
 * overwrites the entries it uses; calls that overlap on the GPU (different
 * streams or threads) race on it, so order them on one stream.
 * Errors: INVALID_ARG, CUDA.  Needs a plan made by tfmm_plan_create. */
tfmm_status tfmm_planewave_noalloc(const tfmm_plan* plan, const double* khat, const double* pol, int32_t R,
                                   tfmm_cfloat* V, void* stream);

/* ------------------------------------------------------------ runtime */

/* Waits for the work queued on `stream` and reports kernel-side failures:
 * TFMM_CUDA if a tensor-core tile gave up waiting on its own copies or MMAs
 * since the plan was made (those outputs are then invalid).  No counterpart in
 * the paper. */
tfmm_status tfmm_sync(tfmm_plan* plan, void* stream);

/* RWG -> (group, slot) table: for every RWG n < n_rwg (mesh order),
 * group[n] is its box group (Sec. II.A) and slot[n] its position in that
 * group's member list (tfmm_plan_members).  Host arrays of n_rwg int32. */
tfmm_status tfmm_plan_rwg_perm(const tfmm_plan* plan, int32_t* group, int32_t* slot);

/* Plan checkpoints.  tfmm_plan_save writes the grid, groups, geometry and the
 * FP64 Tucker factors (Eq. 6) to `path`; tfmm_plan_load rebuilds a plan from
 * such a file on the current device without repeating the setup (the dense
 * tensors of keep_dense are not stored).  A file that is not a checkpoint of
 * this build, is truncated, or holds inconsistent sizes, ranks, members or
 * non-finite factors gives TFMM_IO.  The format is native little-endian. */
tfmm_status tfmm_plan_save(const tfmm_plan* plan, const char* path);
tfmm_status tfmm_plan_load(const char* path, void* stream, tfmm_plan** out);

/* CUDA graphs of the hot path.  Captures stages (1 = aggregate x -> spectra,
 * 2 = disaggregate spectra -> y, 3 = both, in that order) with the given
 * device buffers and arguments (as tfmm_aggregate / tfmm_disaggregate), after
 * running them once eagerly so that first-use allocations stay outside the
 * graph; that eager pass writes the outputs (and applies beta to y).
 * tfmm_graph_launch replays the graph on `stream`: the same buffers are read
 * and written on every replay.  A graph must be destroyed before its plan
 * (tfmm_plan_destroy refuses while graphs exist); replays follow the plan's
 * one-stream ordering rule. */
typedef struct tfmm_graph tfmm_graph;
tfmm_status tfmm_graph_capture(tfmm_plan* plan, int32_t stages, const tfmm_cfloat* x, int32_t R, int64_t ldx,
                               tfmm_cfloat* spectra, int32_t apply_weights, tfmm_cfloat beta, tfmm_cfloat* y,
                               int64_t ldy, tfmm_graph** out);
tfmm_status tfmm_graph_launch(tfmm_graph* graph, void* stream);
tfmm_status tfmm_graph_destroy(tfmm_graph* graph);

/* Tuning of the hot path.  Single RHS: threads per CTA (64..512, multiple of
 * 32), CTAs per SM (0 = as many as fit) and the work-queue order (0 = most
 * factor bytes first, 1 = group order) of the persistent aggregation and
 * disaggregation kernels.  R > 1: the engine (mrhs_precision as in
 * tfmm_params) and two tile shapes of the tensor-core chain.  Changing the
 * tile shapes rebuilds the chains' tile lists (INVALID_ARG while captured
 * graphs of the plan exist). */
typedef struct {
    int32_t agg_threads, agg_ctas_per_sm, agg_order;
    int32_t dis_threads, dis_ctas_per_sm, dis_order;
    int32_t agg_blocks, dis_blocks; /* resulting persistent grids (ignored by _set) */
    int32_t mrhs_precision;
    int32_t tc_f34_n1;              /* tensor cores: cap on r_theta x RHS per CTA of the fused
                                       AG3+AG4 kernel, 0 or 16..256 (0: the largest that fits) */
    int32_t tc_dg1a_pairs;          /* tensor cores: (i_phi, r) pairs per CTA of DG1a, 0, 64 or 128
                                       (0: 128 when it fits, else 64) */
    int32_t single_rhs_split;       /* single-RHS stages as three launches that spread every work
                                       item over many CTAs (for plans with few, large groups):
                                       0 automatic (fewer work items than 2 x SMs), 1 always, 2 never */
    double agg_ms, dis_ms;          /* times the autotuner measured (0 if not tuned) */
} tfmm_tuning;
tfmm_status tfmm_plan_tuning_get(const tfmm_plan* plan, tfmm_tuning* t);
tfmm_status tfmm_plan_tuning_set(tfmm_plan* plan, const tfmm_tuning* t, void* stream);

/* Autotuner: times candidate settings on the plan's own factors with scratch
 * inputs (allocated and freed here; CUDA events on `stream`) and keeps the
 * fastest.  R == 1 searches launch shape and queue order of each stage; R > 1
 * chooses the engine among the 3-term tensor-core chain, the FP32 CUDA-core
 * chain and the single-RHS kernels column by column (and the 2-term chain
 * when allow_two_term != 0, which is less accurate), then, for a tensor-core
 * engine, the two tile shapes of tfmm_tuning.  The search stops early
 * once budget_ms of wall time is spent.  `out` (may be NULL) receives the
 * chosen tuning.  No counterpart in the paper. */
tfmm_status tfmm_autotune(tfmm_plan* plan, int32_t R, double budget_ms, int32_t allow_two_term, void* stream,
                          tfmm_tuning* out);

/* Test hook for the error paths (no counterpart in the paper): the nth device
 * allocation the library makes from now on, on any thread, fails as if the device
 * were out of memory, so the call that makes it returns TFMM_OOM; 0 disarms it.
 * Every plan resource is owned by the plan or by a scoped buffer, so a failed call
 * leaves no device memory behind.  Errors: INVALID_ARG for nth < 0. */
tfmm_status tfmm_test_fail_allocation(int64_t nth);

#ifdef __cplusplus
}
#endif

#endif /* TFMM_H */
