/*
 * afem_mctdhf.h - C ABI of the GB300 (sm_103a) library for MCTDHF on an
 * adaptive finite-element mesh (Orimo, Sato, Ishikawa, arXiv 2301.02387).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns an int status: AFEM_OK (0) or one of the AFEM_E*
 *    codes below.  A human-readable message for the last failure on the
 *    calling host thread is returned by afem_last_error().  No entry point
 *    traps, aborts or exits; device loops carry iteration caps and report
 *    through the status.
 *  - "device" pointers are CUDA global-memory addresses on the device that was
 *    current when the mesh was created; they are owned by the caller and must
 *    stay valid until the work queued on `stream` has finished.  "host"
 *    pointers are ordinary CPU memory owned by the caller.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is queued asynchronously on it unless stated otherwise.
 *  - Vectors over the global unknowns are DoF-major: element (k, v) of an
 *    [N][n_vec] array is at offset k * n_vec + v.  Complex values are
 *    interleaved (re, im) float64 pairs (complex128).
 *  - Global unknowns ("masters") are numbered interior-first: indices
 *    [0, n_interior) are the masters inside the box, [n_interior, N) the
 *    masters on the box surface.  Within each group the order follows the
 *    Morton (Z-order) traversal of the leaf cells.
 *  - The library owns the mesh object and every internal workspace; it
 *    allocates device memory only inside afem_mesh_create and the
 *    workspace-reserving calls documented below.
 */
#ifndef AFEM_MCTDHF_H
#define AFEM_MCTDHF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AFEM_OK 0
#define AFEM_EINVAL 1         /* bad argument: shape, degree, null pointer, kind */
#define AFEM_ENOMEM 2         /* device or host allocation failed */
#define AFEM_ECUDA 3          /* a CUDA runtime call failed */
#define AFEM_EMESH 4          /* mesh construction failed (constraint chain, size limits) */
#define AFEM_ECG_MAXIT 5      /* Poisson CG hit its iteration cap before rtol */
#define AFEM_EBREAKDOWN 6     /* Arnoldi happy breakdown (informational; result valid) */
#define AFEM_ESINGULAR 7      /* one-body density matrix singular */
#define AFEM_ENAN 8           /* a non-finite value was detected */

#define AFEM_MAX_NUCLEI 8

/* Arithmetic forms.  AFEM_PREC_FP64: everything in float64 / complex128.
 * AFEM_PREC_MIXED: the cell operators (stiffness in the Poisson CG sweeps,
 * the packed orbital operator G) run in float32 / complex64; the Poisson
 * solution is refined with float64 residuals to the requested rtol; the
 * two-electron integrals run on the tensor cores (TF32 operands split hi/lo
 * for float32 accuracy, float64 sums of 32-point tiles); and the
 * Arnoldi Gram-Schmidt, the small Krylov exponential, the density-matrix
 * inverse and the CI propagation stay float64. */
#define AFEM_PREC_FP64 0
#define AFEM_PREC_MIXED 1

/* Mesh description (Sec. 3.1 and Sec. 4 of the paper).
 *
 * The box [lo, hi]^3 is covered by n_coarse^3 cubes (the coarse uniform
 * cells); a leaf of level l (side h_l = (hi - lo) / n_coarse / 2^l) is halved
 * while some nucleus a with l < nuc_levels[a] lies within distance
 * refine_c * h_l of the closed cell; the leaves are then 2:1 balanced across
 * faces, edges and vertices.  The paper selects cells with Kelly's error
 * indicator on the nuclear Coulomb potential; this geometric rule stands in
 * for it.  Each leaf carries the tensor-product Lagrange basis of degree
 * `degree` (1..4) through the Gauss-Lobatto points; continuity across
 * coarse/fine interfaces is enforced by hanging-node constraints (the paper's
 * "bridged" functions). */
typedef struct afem_mesh_desc {
    double lo, hi;                          /* box [lo, hi]^3, bohr */
    int32_t n_coarse;                       /* coarse cells per axis (1..1024) */
    int32_t degree;                         /* polynomial degree p (1..4) */
    int32_t n_nuclei;                       /* 0..AFEM_MAX_NUCLEI */
    int32_t pad0;
    double nuc_pos[AFEM_MAX_NUCLEI][3];     /* nucleus positions, bohr */
    double nuc_charge[AFEM_MAX_NUCLEI];     /* nuclear charges Z_a */
    int32_t nuc_levels[AFEM_MAX_NUCLEI];    /* refinement levels L_a toward each nucleus */
    double refine_c;                        /* refinement radius in units of the cell side */
    int32_t refine_mode;                    /* AFEM_REFINE_GEOMETRIC (0) or AFEM_REFINE_KELLY (1) */
    int32_t kelly_max_level;                /* Kelly: finest level (smallest cell h0 / 2^level), 0..12 */
    double kelly_threshold;                 /* Kelly: split a leaf while eta_K > threshold (> 0) */
} afem_mesh_desc;
/* Refinement rules.  AFEM_REFINE_GEOMETRIC: a leaf of level l is split while
 * some nucleus a with l < nuc_levels[a] lies within refine_c * h_l of the
 * closed cell.  AFEM_REFINE_KELLY (Sec. 3.1): every round splits each leaf
 * below kelly_max_level whose Kelly indicator on the nuclear Coulomb potential
 * exceeds kelly_threshold, eta_K^2 = (h_K / 24) sum over its faces of
 * int_F [d_n V_h]^2 (V_h the cellwise interpolant of V = -sum Z_a / |r - R_a|
 * at the cell's GLL nodes, at a node on a nucleus with 1/|r| replaced by its
 * mean over a cube of the node's GLL volume; a coarser or equal neighbour leaf covers the whole
 * face, four finer ones a quarter each; (p+1)^2-point Gauss-Legendre rule per
 * (sub)face; no term on the box surface; a leaf whose closed box contains a
 * nucleus counts as above any threshold), until no leaf splits.  Both rules
 * end with 2:1 balance across faces, edges and vertices (Kelly: after every
 * round). */
#define AFEM_REFINE_GEOMETRIC 0
#define AFEM_REFINE_KELLY 1

typedef struct afem_mesh_info {
    int64_t n_cells;        /* leaf cells */
    int64_t n_masters;      /* global unknowns N (interior + surface) */
    int64_t n_interior;     /* masters inside the box (orbital unknowns) */
    int64_t n_hanging;      /* constrained support points */
    int64_t n_constraint_entries; /* nonzeros of the hanging rows of C */
    int32_t degree;
    int32_t max_level;
    double h_min, h_max;    /* smallest / largest leaf side */
} afem_mesh_info;

typedef struct afem_mesh afem_mesh;   /* opaque */

/* Message describing the last failure on this host thread ("" if none). */
const char* afem_last_error(void);

/* Number of CUDA kernels this library has launched in this process so far
 * (host-side counter, all devices and threads).  Library bookkeeping with no
 * counterpart in the paper. */
int afem_kernel_launch_count(int64_t* count);

/* The binary64 <-> binary32 conversions of the precision form (library
 * arithmetic with no counterpart in the paper), applied to n device values:
 * AFEM_CONVERT_F64_F32 rounds x (double[n]) to nearest-even into y (float[n]),
 * AFEM_CONVERT_F32_F64 widens x (float[n]) exactly into y (double[n]).  They
 * follow the IEEE-754 bit layouts on the integer pipe instead of the
 * hardware conversions (which issue on GB300's FP64 pipe); values outside the
 * binary32 normal range map to signed zeros (below, including binary32
 * subnormal inputs) or infinities (above).  Exposed so that tests can compare
 * them with the hardware conversions.  Asynchronous on `stream`; x and y are
 * caller-owned and must not overlap.  Errors: AFEM_EINVAL (n < 0, null
 * buffers with n > 0, unknown direction), AFEM_ECUDA. */
#define AFEM_CONVERT_F64_F32 0
#define AFEM_CONVERT_F32_F64 1
int afem_convert(const void* x, void* y, int64_t n, int direction, void* stream);

/* Kernel-class timing (library instrumentation with no counterpart in the
 * paper).  While enabled (process-wide), the library brackets each call of a
 * class's kernels with a pair of CUDA events recorded on the stream the
 * kernels are launched on, and adds the call's algorithmic work: FP64 flops
 * for AFEM_PROF_GS (8 per complex multiply-add with a Krylov vector, 4 per
 * squared norm) and AFEM_PROF_CELL64 (3 (p+1) 2 + 6 per node and real
 * column), bytes for the others (each input and output element once).
 * afem_profile_read waits for the recorded events of class `cls` and returns
 * (each pointer may be NULL) the summed event time in milliseconds, the
 * number of bracketed calls and the summed work; reset != 0 clears the class
 * afterwards.  Errors: AFEM_EINVAL (unknown class), AFEM_ECUDA. */
#define AFEM_PROF_GS 0      /* Arnoldi Gram-Schmidt passes (FP64)            */
#define AFEM_PROF_GCELL32 1 /* complex64 cell pass of G (precision form)     */
#define AFEM_PROF_STIFF32 2 /* float32 stiffness of the CG sweeps            */
#define AFEM_PROF_CGVEC32 3 /* float32 CG vector kernels                     */
#define AFEM_PROF_CELL64 4  /* FP64 cell passes (G and stiffness)            */
#define AFEM_PROF_COUNT 5
int afem_profile_enable(int on);
int afem_profile_read(int cls, double* ms, int64_t* calls, double* work, int reset);

/* Measured arithmetic peak of the current device (library instrumentation
 * with no counterpart in the paper): fused multiply-add throughput in FP64
 * (AFEM_PEAK_FP64) or FP32 (AFEM_PEAK_FP32), in flop/s (2 per multiply-add),
 * from 4 blocks of 256 threads per SM, each thread running 8 independent
 * multiply-add chains.  The loop length is calibrated so that one launch
 * takes about target_ms (0 < target_ms <= 1e4); the best of 3 timed launches
 * (CUDA events on `stream`) is returned in *flops_per_s.  Allocates and frees
 * one scalar of device memory; synchronous.  Errors: AFEM_EINVAL (unknown
 * kind, target out of range, null output), AFEM_ECUDA. */
#define AFEM_PEAK_FP64 0
#define AFEM_PEAK_FP32 1
int afem_fma_peak(int kind, double target_ms, double* flops_per_s, void* stream);

/* Build the mesh on the host and upload every table to the current device.
 * Sec. 3.1 (coarse cubes halved toward the nuclei; GLL tensor basis; bridged
 * functions).  *out receives a library-owned object; free it with
 * afem_mesh_destroy.  Returns AFEM_EINVAL for a bad description, AFEM_EMESH
 * if a hanging point would be constrained by another hanging point (cannot
 * happen after 2:1 balance), AFEM_ENOMEM / AFEM_ECUDA on device failures.
 * Synchronous. */
int afem_mesh_create(const afem_mesh_desc* desc, afem_mesh** out);

/* As afem_mesh_create, but with flags.  AFEM_MESH_HOST_ONLY builds the host
 * tables only (no device allocation, no CUDA call): afem_mesh_get_info and
 * afem_mesh_tables work, every device entry point returns AFEM_EINVAL.  Used
 * to inspect meshes on machines without a GPU.  Synchronous. */
#define AFEM_MESH_HOST_ONLY 1
int afem_mesh_create_ex(const afem_mesh_desc* desc, int flags, afem_mesh** out);

/* Release the mesh and its device tables.  NULL is accepted.  Synchronous. */
int afem_mesh_destroy(afem_mesh* mesh);

/* Kernel-shape options of a mesh (library tuning; no counterpart in the paper).
 * AFEM_OPT_CELL32_VARIANT selects the float32 four-lane cell pass: 0 (default)
 * computes each output node in one thread, 1 computes the 1D contractions
 * line by line with direction-wise accumulation in shared memory, 2 does the
 * same for the stiffness with one thread per (line, column pair) and the 1D
 * matrix in registers (1, 2 or 4 column quads; other passes as for 0).  All
 * give the same operator up to float rounding order.  Host only. */
#define AFEM_OPT_CELL32_VARIANT 1
/* AFEM_OPT_POISSON_SOLVER selects the preconditioner of the batched Poisson
 * CG (Sec. 3.1 solves the mean fields by CG with algebraic multigrid):
 * AFEM_POISSON_JACOBI (default) or AFEM_POISSON_MULTIGRID, a geometric
 * multigrid V-cycle over the mesh at degrees p, p/2, .., 1 and then degree 1
 * on the octree truncated at levels L-1, .., 0 (every leaf finer than the cap
 * replaced by its ancestor there; so for meshes of either refinement rule)
 * (exact interpolation between the nested spaces, restriction its transpose,
 * Chebyshev-Jacobi smoothing of degree 3, a degree-30 Chebyshev polynomial on
 * the uniform coarse grid).  The FP64 form runs CG with the float64 V-cycle;
 * the precision form runs float64 defect correction whose corrections are
 * float32 CG iterations with the float32 V-cycle.  The hierarchy (its meshes,
 * transfer tables and eigenvalue estimates) is built on the first solve and
 * kept by the mesh.  Same stopping test, same result to rtol. */
#define AFEM_OPT_POISSON_SOLVER 2
#define AFEM_POISSON_JACOBI 0
#define AFEM_POISSON_MULTIGRID 1
/* AFEM_OPT_GCELL_BLOCKS (degree-4 meshes, even orbital counts, precision
 * form, length gauge, no complex scaling): 1 (default) forms, once per
 * orbital propagation, the frozen pointwise part of G at every cell node,
 * m_node (U_pq + delta_pq (V + E.x)), as one contiguous block per cell, which
 * the float32 G cell pass stages into shared memory with one bulk copy
 * (cp.async.bulk, the tensor memory accelerator) instead of gathering the
 * mean-field rows node by node; 0 gathers them (and forms the potential term)
 * inside the pass; 2 (n <= 4) runs the blocks in a persistent, double-buffered
 * loop over cells (the next cell's copies in flight while a cell is computed,
 * v at the hanging points formed first), measured slower than 1 on GB300.
 * Same operator in every form (float32 rounding aside). */
#define AFEM_OPT_GCELL_BLOCKS 3
int afem_mesh_set_option(afem_mesh* mesh, int option, int value);

/* Exterior complex scaling of the kinetic energy (Sec. 4: an absorbing
 * boundary by ECS outside an inner box; the paper leaves the construction to
 * its references).  Built: Cartesian scaling with a sharp onset at the faces of
 * the inner box |x_d| <= half_width[d], x_d -> +-R_d + e^{i theta} (x_d -+ R_d)
 * outside.  A cell outside the box along the axes with flag f_d has
 * eta_d = e^{i theta f_d}, J = prod_d eta_d, the weak-form stiffness
 * h sum_d (J / eta_d^2) (d-th Kronecker term) and the mass J h^3 W (x) W (x) W;
 * with M_theta = C^T (J m_f) the kinetic operator becomes
 * 1/2 M_theta^-1 A_theta.  The nuclear potential, E . r and the mean fields
 * keep their real weights; the orbital inner product stays u^H M_L v.  Every
 * one-body operator of the orbital path then uses it: AFEM_OP_H1 and
 * AFEM_OP_H1_C64, afem_arnoldi_step / _propagate and afem_mctdhf_step (whose
 * h_pq and CI Hamiltonian become non-Hermitian).  Not built with it (AFEM_EINVAL):
 * the velocity gauge, imaginary-time steps, the afem_tdse_* adjoint, the batch.
 * theta in [0, pi/2); theta = 0 removes the scaling.  Every cell must lie wholly
 * inside or outside the box along each axis (else AFEM_EMESH).  The current
 * device must be the mesh's.  Host set-up plus a synchronous upload of per-cell
 * flags and per-master factors M_L / M_theta (library-owned). */
int afem_mesh_set_ecs(afem_mesh* mesh, double theta, const double half_width[3]);

/* Sizes of the mesh (host struct, caller-owned). */
int afem_mesh_get_info(const afem_mesh* mesh, afem_mesh_info* info);

/* Copy mesh tables to caller-owned HOST buffers (any pointer may be NULL to
 * skip it).  coords: [N][3] master coordinates; lumped_mass: [N] lumped mass
 * M_L = C^T m_f (Sec. 3.1, mass matrix with GLL quadrature, row-summed at
 * hanging masters); cells: [n_cells][4] (level, i, j, k) of each leaf in the
 * library's cell order. */
int afem_mesh_tables(const afem_mesh* mesh, double* coords, double* lumped_mass,
                     int32_t* cells);

/* Operator kinds for afem_op_apply. */
#define AFEM_OP_H1 0      /* y = M_L^{-1} H1~ x, complex128, Dirichlet (Eq. discretized_eom) */
#define AFEM_OP_STIFF 1   /* y = A x, float64, full Neumann stiffness over all masters */
#define AFEM_OP_STIFF_F32 2  /* as AFEM_OP_STIFF in float32 (precision form) */
#define AFEM_OP_H1_C64 3     /* as AFEM_OP_H1 in complex64 (precision form) */
#define AFEM_OP_POS 4        /* y = M_L^{-1} F[e.r] x, complex128, Dirichlet: the position operator
                                along e (passed as E); dipole and field derivative of H1~ */
#define AFEM_OP_FORCE 5      /* y = M_L^{-1} F[e.f] x, complex128, Dirichlet, f = -grad V the nuclear
                                force on an electron (0 at a support point on a nucleus): the
                                potential part of the Ehrenfest acceleration along e (passed as E) */
#define AFEM_OP_H1_VG 6      /* y = M_L^{-1} H1~(A) x, complex128, Dirichlet: the velocity-gauge one-body
                                Hamiltonian of Sec. 2 with the vector potential A passed as E */
#define AFEM_OP_H1_VG_C64 7  /* as AFEM_OP_H1_VG in complex64 (precision form) */

/* Matrix-free operator application on n_vec vectors at once (Sec. 3.1).
 *
 * AFEM_OP_H1: H1~ = 1/2 A + F[V + E.r] is the length-gauge one-body
 *   Hamiltonian matrix (H1)_kl = int b_k H1 b_l with GLL quadrature, V the
 *   nuclear Coulomb potential; x and y are complex128 [N][n_vec] device
 *   arrays.  Surface entries of x are treated as zero and surface entries of
 *   y are written as zero (orbitals vanish on the box surface).  E is a host
 *   array of 3 doubles (field in a.u.); NULL means zero field.
 * AFEM_OP_H1_VG: H1~(A) = 1/2 A + F[V] - i sum_d A_d G_d, the velocity gauge
 *   of Sec. 2 (H1 = -1/2 Laplacian + V - i A(t) . grad; the A^2/2 term is a
 *   global phase and is left out), with G_d = C^T (sum_K P_K^T h_K^2
 *   (W (x) W (x) S)_d P_K) C the skew-symmetric form of int b_k d_d b_l,
 *   S = (Dw - Dw^T) / 2, Dw[i][j] = w_i L_j'(xi_i): it equals the plain form on
 *   conforming cells and keeps H1~(A) Hermitian across hanging faces.  A is
 *   passed in E (NULL: A = 0).
 * AFEM_OP_STIFF: A = C^T (sum_K P_K^T A_K P_K) C with the GLL cell stiffness
 *   A_K; x and y are float64 [N][n_vec] device arrays; E is ignored.
 * n_vec: 1..64.  x and y must not overlap.  Asynchronous on `stream`. */
int afem_op_apply(afem_mesh* mesh, int kind, const double* E, const void* x, void* y,
                  int n_vec, void* stream);

/* Mean-field potentials of all orbital pairs by batched Poisson solves
 * (Sec. 3.1: Delta W^r_s = -4 pi phi_r^* phi_s, Dirichlet data = the direct
 * integral of Eq. mean-field on the box surface, solved by CG).
 *
 * phi: complex128 [N][n_orb] device array of orbital nodal values (surface
 *   entries are treated as zero).  n_orb: 1..8.
 * W: float64 [N][n_orb^2] device array, in/out.  Column c holds the real
 *   potential of density column c: c < n_orb is |phi_c|^2; then, for each
 *   pair r < s in row-major order, Re and Im of conj(phi_r) phi_s.  The
 *   complex W^r_s is (Re column) + i (Im column), W^s_r its conjugate.
 *   On return the surface rows hold the Dirichlet data (multipole expansion
 *   about the box centre, l <= 12) and the interior rows the CG solution.
 *   warm_start != 0 starts CG from the interior rows passed in.
 * Jacobi-preconditioned CG per column; column c stops when
 *   ||r_c|| <= rtol ||b_c - A_IB g_c||.  iters_out (host, may be NULL)
 *   receives the iterations run; relres_out (host [n_orb^2], may be NULL) the
 *   final relative residuals.
 * Returns AFEM_ECG_MAXIT if some column has not converged after max_it
 * iterations (W holds the last iterate), AFEM_ENAN on non-finite residuals.
 * Allocates (grow-only) device workspace owned by the mesh on first use.
 * Synchronises `stream` every few iterations to test convergence. */
int afem_poisson_batch(afem_mesh* mesh, const void* phi, int n_orb, void* W, double rtol,
                       int max_it, int warm_start, int* iters_out, double* relres_out,
                       void* stream);

/* As afem_poisson_batch with a choice of arithmetic.  AFEM_PREC_MIXED runs one
 * Jacobi-PCG per column in float32 (operator, vectors) on the residual scaled
 * to unit norm, folds its correction into the float64 W, and replaces the
 * float32 residual by the true float64 residual (rescaling the search
 * direction) whenever the float32 residual has dropped 100-fold since the last
 * replacement or claims convergence ("reliable updates").  It stops on the
 * same float64 test as afem_poisson_batch.  iters_out counts float32
 * iterations (bounded by max_it), outer_out (host, may be NULL) the float64
 * residual evaluations. */
int afem_poisson_batch_ex(afem_mesh* mesh, const void* phi, int n_orb, void* W, double rtol,
                          int max_it, int warm_start, int precision, int* iters_out,
                          int* outer_out, double* relres_out, void* stream);

/* Surface data of the pair mean fields without any device allocation.
 *
 * The paper has no counterpart: this is a library service.  It computes the
 * same Dirichlet data as afem_poisson_batch (multipole expansion about the
 * box centre, l <= 12, of every pair density of phi) and writes it into the
 * surface rows [n_interior, N) of W (float64 [N][n_orb^2], same column
 * layout); interior rows are not touched.  phi: complex128 [N][n_orb].
 *
 * It exists for callers that must not allocate device memory once they are
 * running: for example a process whose device memory is fully reserved by
 * another allocator's pool, or a service loop with a fixed memory budget.
 * Such callers cannot use afem_poisson_batch, which grows a workspace on first
 * use.  Here the scratch (moment partials and moments) is one file-scope
 * device array of 413,712 doubles (about 3.2 MiB), held by every GPU that
 * loads the library until the process exits; nothing is allocated or freed.
 *
 * Limits and behaviour:
 *  - n_orb must be 1..AFEM_NOALLOC_MAX_ORB; larger values return AFEM_EINVAL.
 *  - The current device must be the mesh's device (else AFEM_EINVAL).
 *  - The first call on a device looks up the device address of the scratch
 *    array (with that device current) and uploads the solid-harmonic
 *    constants of the expansion (two synchronous copies); make that first
 *    call before any stream capture.
 *  - All calls share the one scratch array and each call overwrites it
 *    completely before reading it; calls that overlap on the GPU (other
 *    streams, other host threads) race and must be serialised by the caller.
 * Asynchronous on `stream`. */
#define AFEM_NOALLOC_MAX_ORB 4
int afem_poisson_boundary_noalloc(afem_mesh* mesh, const void* phi, int n_orb, void* W, void* stream);

/* Two-electron integrals of orbitals phi with their pair mean fields W (Sec. 2,
 * the integrals of Eq. ci_eom with the potentials of Eq. mean-field):
 *   (pq|rs) = sum_f m_f conj(phi_p(f)) phi_q(f) W^r_s(f)
 * over every support point f (hanging points through the constraints C), m_f
 * the assembled GLL weight.  The same quantity the MCTDHF step forms.
 * phi: complex128 [N][n_orb] device (surface entries treated as zero);
 * W: float64 [N][n_orb^2] device in the column layout of afem_poisson_batch;
 * eri: complex128 [n_orb^2][n_orb^2] device, caller-owned, written
 *   eri[(p n + q) n^2 + (r n + s)] = (pq|rs).  n_orb: 1..8.
 * precision: AFEM_PREC_FP64 (float64 sums) or AFEM_PREC_MIXED (the contraction
 *   as tcgen05 tensor-core MMAs: TF32 operands split hi/lo, three products per
 *   tile, float32 sums of 32 support points added in float64).
 * Allocates (grow-only) device workspace owned by the mesh on first use.
 * Synchronises `stream` (reads a status word); AFEM_ECUDA if a tensor-core
 * block gave up waiting for its MMAs (bounded waits; no hang). */
int afem_two_electron_integrals(afem_mesh* mesh, const void* phi, int n_orb, const void* W, void* eri,
                                int precision, void* stream);

/* One short-iterative Arnoldi step of the packed orbital equation with the
 * operator frozen (Sec. 3.2, Eq. packed_orb_eom; Eq. orb_eom with X = 0):
 *   (G v)_p = Q [ M_L^-1 ( H1~ v_p + C^T diag(m_f) sum_q (C U_pq) o (C v_q) ) ],
 *   Q y = y - sum_j phi_j (phi_j^H M_L y),
 *   phi_out = beta V_m exp(-i dt H_m) e_1   (Arnoldi in the inner product
 *   <u,v> = sum_p u_p^H M_L v_p, beta = ||phi||; each new vector is
 *   orthogonalised by classical Gram-Schmidt -- all inner products in one
 *   pass, the update in a second -- and by a second such pair of passes only
 *   when the update left less than 1e-2 of the vector's norm).
 * phi, phi_out: complex128 [N][n_orb] device arrays (must not alias).
 * U: complex128 [N][n_orb][n_orb] device array of mean-field operator
 *   fields U_pq = sum_o (D^-1)^o_p sum_rs P^{qs}_{or} W^r_s at the masters,
 *   or NULL for no mean field.  E: host double[3] field (NULL = 0).
 * krylov_m: 1..16.  err_est (host, may be NULL): beta |h_{m+1,m}|
 *   |e_m^T exp(-i dt H_m) e_1|, 0 after a happy breakdown; m_used and
 *   breakdown (host, may be NULL) report the dimension actually used.
 * Allocates (grow-only) mesh-owned workspace; synchronises `stream` once,
 * after the Krylov space is built (the breakdown test reads the Hessenberg
 * matrix on the host). */
int afem_arnoldi_step(afem_mesh* mesh, const double* E, const void* phi, const void* U, int n_orb,
                      int krylov_m, double dt, void* phi_out, double* err_est, int* m_used,
                      int* breakdown, void* stream);

/* As afem_arnoldi_step with a choice of arithmetic.  AFEM_PREC_MIXED applies
 * the cell pass of G in complex64 to a complex64 copy of each Krylov vector
 * (and of U); the projector overlaps, the projection, Gram-Schmidt, the small
 * exponential and the combination stay complex128. */
int afem_arnoldi_step_ex(afem_mesh* mesh, const double* E, const void* phi, const void* U, int n_orb,
                         int krylov_m, double dt, int precision, void* phi_out, double* err_est,
                         int* m_used, int* breakdown, void* stream);

/* exp(-i G dt) phi with error control (Sec. 3.2): G frozen as in
 * afem_arnoldi_step; dt is covered by substeps tau_1, tau_2, ..., each from a
 * fresh Krylov space of dimension krylov_m built from the current vector.
 * Each substep is the longest of the candidates tau_max 2^(-c/8), c = 0..63,
 * whose estimate beta |h_{m+1,m}| |e_m^T exp(-i tau H_m) e_1| is <= tol *
 * beta, with tau_max the whole remainder for the first substep and
 * min(remainder, 2 tau_previous) after it; when no candidate passes, the
 * candidates continue below the smallest one (at most 8 more sets of 64, then
 * the smallest is taken).  The 64 candidate exponentials are evaluated in one
 * launch.  A breakdown takes the whole remainder exactly.  tol <= 0: one step
 * over dt.  err_est (host, may be NULL) receives the sum of the accepted
 * estimates, substeps (host, may be NULL) the substep count.  More than 4096
 * substeps returns AFEM_EINVAL.  Allocates (grow-only) mesh-owned workspace;
 * synchronises `stream` once per substep. */
int afem_arnoldi_propagate(afem_mesh* mesh, const double* E, const void* phi, const void* U, int n_orb,
                           int krylov_m, double dt, int precision, double tol, void* phi_out,
                           double* err_est, int* substeps, void* stream);

/* exp(-i G dt) phi by the rule of Sec. 3.2 (the dimension of the Krylov space
 * is chosen by the error estimate at a fixed step): dt is split into `steps`
 * (1..4096) equal steps tau = dt / steps; in each, the Arnoldi process of
 * afem_arnoldi_step adds one vector at a time and, after vector j + 1,
 * evaluates beta |h_{j+2,j+1}| |e_{j+1}^T exp(-i tau H_{j+1}) e_1|; the first
 * dimension whose estimate is <= tol * beta is used (a breakdown uses the
 * exact projected exponential); if none up to m_max (1..16) is, m_max is used
 * and the step is counted in *unmet.  err_est, dim_max, dim_sum, unmet (host,
 * each may be NULL): the summed estimates, the largest and the summed
 * dimensions, the unmet steps.  Allocates (grow-only) mesh-owned workspace;
 * synchronises `stream` once per added vector.  Errors: AFEM_EINVAL
 * (arguments), AFEM_ENAN, AFEM_ENOMEM, AFEM_ECUDA. */
int afem_arnoldi_adaptive(afem_mesh* mesh, const double* E, const void* phi, const void* U, int n_orb,
                          int m_max, double dt, int steps, int precision, double tol, void* phi_out,
                          double* err_est, int* dim_max, int* dim_sum, int* unmet, void* stream);

/* MCTDHF time stepper (Sec. 2 and Sec. 3.2): owns the determinant-space
 * tables and its device workspace; the mesh must outlive it. */
typedef struct afem_mctdhf afem_mctdhf;

typedef struct afem_step_info {
    double energy;          /* electronic energy at t: sum h_pq gamma_pq + 1/2 sum (pq|rs) Gamma_pqrs */
    double arnoldi_err;     /* Krylov error estimate of the orbital step */
    double cg_relres_max;   /* largest final relative residual of the Poisson batch */
    int32_t krylov_m_used;
    int32_t breakdown;
    int32_t cg_iters;
    int32_t krylov_substeps; /* Krylov substeps taken (1 unless a Krylov tolerance is set) */
    double dipole[3];        /* <sum_i r_i> at t: sum_pq gamma_pq phi_p^H F[x_d] phi_q, d = x, y, z
                                (summed electron positions; the dipole moment is its negative) */
    int32_t krylov_dim_sum;  /* Krylov dimensions summed over the substeps (G applications) */
    int32_t krylov_unmet;    /* adaptive dimension: steps whose estimate stayed above the threshold */
} afem_step_info;

/* n_orb spatial orbitals (1..8), n_alpha / n_beta electrons per spin
 * (0..n_orb each, not both 0), Krylov dimension krylov_m (1..16).  The CI
 * vector holds all determinants: index I = i_alpha * n_beta_strings + i_beta,
 * strings of occupied orbitals ordered by ascending bit mask (bit p =
 * orbital p); |I> = prod_alpha a+ prod_beta a+ |0> in ascending orbital order.
 * Synchronous. */
int afem_mctdhf_create(afem_mesh* mesh, int n_orb, int n_alpha, int n_beta, int krylov_m,
                       afem_mctdhf** out);
int afem_mctdhf_destroy(afem_mctdhf* solver);
/* Arithmetic of later steps: AFEM_PREC_FP64 (default) or AFEM_PREC_MIXED
 * (Poisson by float32 PCG inside float64 refinement, G cell pass in
 * complex64; everything else float64).  Host only, no device work. */
int afem_mctdhf_set_precision(afem_mctdhf* solver, int precision);
/* Krylov accuracy control of later steps (Sec. 3.2: the Krylov propagation
 * is controlled by an a-posteriori error estimate, 1e-10 in the paper).
 * tol = 0 (default): one Krylov step of dimension krylov_m per time step.
 * tol > 0: the orbital step is split into substeps of the same frozen G, each
 * short enough that its estimate stays below tol * ||phi|| (see
 * afem_arnoldi_propagate).  Host only. */
int afem_mctdhf_set_krylov_tol(afem_mctdhf* solver, double tol);
/* The Krylov rule of Sec. 3.2 for later steps: steps > 0 splits each time
 * step into `steps` equal Krylov steps, each with the smallest dimension (up
 * to krylov_m) whose estimate is <= tol ||phi|| (see afem_arnoldi_adaptive;
 * tol from afem_mctdhf_set_krylov_tol, which must then be > 0); 0 (default)
 * returns to the rule of afem_mctdhf_set_krylov_tol.  Host only. */
int afem_mctdhf_set_krylov_adaptive(afem_mctdhf* solver, int steps);
/* Imaginary-time steps for ground-state preparation (Sec. 4 prepares its
 * initial state by imaginary-time propagation; the scheme is this library's
 * reading): on = 1 makes later afem_mctdhf_step calls advance tau by dt with
 * t = -i tau -- the same frozen quantities as the real-time step, then
 * C <- exp(-dt H_CI) C / ||.|| (Taylor series of H_CI - <H_CI>),
 * phi <- exp(-dt G) phi by the Arnoldi process (the Krylov rule set by the
 * functions above, with exp(-tau H_m) in place of exp(-i tau H_m)), and
 * phi <- phi S^-1/2 with S = phi^H M_L phi (Loewdin; the n x n root is
 * formed on the host).  The reported energy is that of the state at the
 * start of the step.  on = 0 (default) returns to real time.  Host only;
 * a step in this mode returns AFEM_ESINGULAR if S is not positive definite. */
int afem_mctdhf_set_imaginary(afem_mctdhf* solver, int on);
/* Gauge of later steps: AFEM_GAUGE_LENGTH (default; the step's E argument is
 * the field E(t), H1 contains E . r) or AFEM_GAUGE_VELOCITY (Sec. 2; the step's
 * E argument is the vector potential A(t) = -int_-inf^t E, H1 contains
 * -i A . grad as in AFEM_OP_H1_VG, in h_pq, in the G cell passes and hence in
 * the energy).  Host only. */
#define AFEM_GAUGE_LENGTH 0
#define AFEM_GAUGE_VELOCITY 1
int afem_mctdhf_set_gauge(afem_mctdhf* solver, int gauge);
/* Number of determinants (host). */
int afem_mctdhf_ci_dim(const afem_mctdhf* solver, int64_t* dim);

/* One time step t -> t + dt with the field E(t) frozen (first order, Sec. 3.2):
 *   W <- pair mean fields of phi(t) (afem_poisson_batch, warm-started from W);
 *   h_pq, (pq|rs), gamma, Gamma at t; C <- exp(-i dt H_CI(t)) C (Eq. ci_eom,
 *   X = 0; Taylor series of H_CI - <H_CI> with 30 terms, accurate while
 *   ||H_CI - <H_CI>|| dt <= 3); phi <- exp(-i G(t) dt) phi by short-iterative
 *   Arnoldi (Eq. packed_orb_eom).
 * phi: complex128 [N][n_orb] device, in/out (surface rows must be zero).
 * C: complex128 [ci_dim] device, in/out.  W: float64 [N][n_orb^2] device,
 *   in/out (column layout of afem_poisson_batch; pass zeros at the first step).
 * E: host double[3] (NULL = 0).  info: host, may be NULL.
 * Returns AFEM_ESINGULAR if the one-body density matrix cannot be inverted
 * (nothing is updated then), AFEM_ECG_MAXIT if the Poisson batch did not reach
 * cg_rtol (the step is still taken with the last iterate).
 * Synchronises `stream` several times per step. */
int afem_mctdhf_step(afem_mctdhf* solver, void* phi, void* C, void* W, const double* E, double dt,
                     double cg_rtol, int cg_max_it, afem_step_info* info, void* stream);

/* Batching form of the time step: one afem_mctdhf_step of each of `count`
 * independent instances (solvers with their own meshes, sizes, degrees,
 * orbital counts and arithmetic forms) per call.  Each instance computes
 * exactly what afem_mctdhf_step computes for it; the batch shares the
 * schedule: instances are spread over W worker streams (longest estimated
 * cost first, instances that share a mesh on one worker), one host thread per
 * stream issues its instances' steps, and the GPU overlaps them.  W is tuned
 * on the batch's own steps: the first call (which allocates workspaces) runs
 * on 4 streams, the next calls each try one of 1, 2, 4, 8, 16 (up to count),
 * and later calls use the fastest (afem_batch_stepper_tuning).
 * solvers: host array of `count` solver handles (caller-owned, kept alive
 *   while the batch exists), all on the current device.
 * phi, C, W: host arrays of `count` device pointers, each as afem_mctdhf_step
 *   takes them; E: host [count][3] fields at t (NULL: field-free).
 * infos: host [count] (may be NULL).  The caller's `stream` is ordered before
 *   and after the batch by events; the call returns when every instance's
 *   step has completed on the GPU.
 * Returns the first hard error (with the instance number in the message),
 * else AFEM_ECG_MAXIT if some instance's Poisson batch hit its limit.
 * Kernel-class timing (afem_profile_enable) must be off during the call. */
typedef struct afem_batch_stepper afem_batch_stepper;
int afem_batch_stepper_create(afem_mctdhf* const* solvers, int count, afem_batch_stepper** out);
int afem_batch_stepper_destroy(afem_batch_stepper* batch);
int afem_batch_stepper_step(afem_batch_stepper* batch, void* const* phi, void* const* C, void* const* W,
                            const double* E, double dt, double cg_rtol, int cg_max_it, afem_step_info* infos,
                            void* stream);
/* streams: the tuned worker count (0 while still tuning); cand_streams /
 * cand_ms (host, n_candidates entries, each may be NULL): the candidates and
 * their measured wall time per batched step. */
int afem_batch_stepper_tuning(const afem_batch_stepper* batch, int* streams, int* n_candidates,
                              int* cand_streams, double* cand_ms);

/* ---- Differentiation form: the one-electron limit of the orbital step.
 * With one orbital and one configuration the mean fields and the projector
 * of Eq. orb_eom vanish and the step is the Schroedinger propagator of the
 * length-gauge H1~ (Sec. 3.1, Sec. 3.2):
 *   phi_{k+1} = exp(-i dt H~(E_k)) phi_k,  H~(E) = M_L^-1 H1~(E e_dir),
 *   d_k = <phi_k, O phi_k>_M,  k = 0..n_steps,
 * for a field E(t) = E_k e_dir held fixed over step k (k < n_steps).  The
 * signal's operator is chosen by `observable`: AFEM_OP_POS, O = Z~ =
 * M_L^-1 F[e_dir . r] (the dipole), or AFEM_OP_FORCE, O = M_L^-1 F[e_dir . f]
 * with f = -grad V (the potential part of the Ehrenfest acceleration, whose
 * full value adds -(e_dir . e_dir) E(t_k) for the electron).  Whatever the
 * observable, dH~/dE = Z~ drives the derivatives.
 * Each step is one afem_arnoldi_propagate without projector (krylov_m, tol
 * and precision as there, except that tol = 0 takes one Krylov step of
 * dimension krylov_m per time step).
 * Arguments common to the three calls: e_dir host [3] (unit field direction;
 * any vector is accepted and scales the field), E host [n_steps] field
 * amplitudes (a.u.), dt > 0, krylov_m 1..16, tol >= 0, precision
 * AFEM_PREC_FP64 or AFEM_PREC_MIXED, observable AFEM_OP_POS or
 * AFEM_OP_FORCE.  All three synchronise `stream` and
 * allocate mesh-owned (grow-only) workspace.  Errors: AFEM_EINVAL (null or
 * out-of-range argument, host-only mesh), AFEM_ENOMEM, AFEM_ECUDA, and the
 * Arnoldi errors.
 *
 * afem_tdse_forward: phi0 complex128 [N] device (surface entries read as 0),
 * n_steps >= 0.  d host [n_steps + 1] receives the dipole signal; phi_end
 * (device [N], may be NULL) the final state.  ckpt (device, may be NULL):
 * complex128 [ceil(n_steps / ckpt_every)][N]; slot c receives phi_{c
 * ckpt_every}; ckpt_every >= 1 when ckpt is given. */
int afem_tdse_forward(afem_mesh* mesh, const double* e_dir, const double* E, int n_steps, double dt,
                      int krylov_m, double tol, int precision, int observable, const void* phi0,
                      void* phi_end, double* d, void* ckpt, int ckpt_every, void* stream);
/* afem_tdse_jvp: the tangent map v -> dd = (dd/dE) v along the trajectory from
 * phi0, by propagating [dphi; phi] with exp(-i dt [[H~, v_k Z~], [0, H~]])
 * (the block form of the Frechet derivative of exp).  v host [n_steps]; d and
 * dd host [n_steps + 1] receive the signal and its directional derivative. */
int afem_tdse_jvp(afem_mesh* mesh, const double* e_dir, const double* E, int n_steps, double dt,
                  int krylov_m, double tol, int precision, int observable, const void* phi0,
                  const double* v, double* d, double* dd, void* stream);
/* afem_tdse_vjp: the adjoint map g -> grad_E = (dd/dE)^T g, n_steps >= 1.
 * ckpt/ckpt_every as written by afem_tdse_forward with the same E, dt,
 * krylov_m, tol and precision; each segment of ckpt_every steps is recomputed
 * from its checkpoint, then swept backward with
 *   [lam_k; mu_k] = exp(+i dt [[H~, 0], [Z~, H~]]) [lam_{k+1}; 0],
 *   grad_E[k] = 2 Re <mu_k, phi_k>_M,  lam_k <- lam_k + g_k O phi_k,
 * from lam_{n_steps} = g_{n_steps} O phi_{n_steps}.  g host [n_steps + 1],
 * grad_E host [n_steps]; lam0 (device complex128 [N], may be NULL) receives
 * lam_0, the gradient with respect to phi0 in <.,.>_M. */
int afem_tdse_vjp(afem_mesh* mesh, const double* e_dir, const double* E, int n_steps, double dt,
                  int krylov_m, double tol, int precision, int observable, const void* ckpt,
                  int ckpt_every, const double* g, double* grad_E, void* lam0, void* stream);

/* ---- Batching form: many independent instances in one launch.
 * The FP32 cell passes of Sec. 3.1 (Eq. discretized_eom) applied to every
 * instance of a batch of meshes (uneven sizes, degrees 1..4) by one persistent
 * kernel: for each instance i, y_i = M_L^-1 H1~(E_i) x_i with Dirichlet rows
 * zero (AFEM_OP_H1_C64: x_i, y_i complex64 [N_i][n_vec_i]) or y_i = A x_i
 * (AFEM_OP_STIFF_F32: float32 [N_i][n_vec_i]), the same result as
 * afem_op_apply on that mesh up to the order of the floating-point atomic
 * sums.  The persistent kernel moves each node's values as 16-byte quads; a
 * batch with an instance whose values are not whole quads (an odd orbital
 * count, real columns not a multiple of 4, or a buffer not 16-byte aligned)
 * runs the per-instance schedule below only.  Small cells (p <= 3, few quads) are grouped
 * into work items that fill a block.  The first apply of a (kind, n_vec)
 * signature times candidate schedules on the batch itself -- the persistent
 * launch with grids of 2 or all resident blocks per SM at 256 and 128
 * threads or one block per work item, and the instances' own passes on 4, 8
 * or 16 parallel streams (reported as block 0, grid = streams) -- and keeps
 * the fastest (afem_batch_get_tuning).  With
 * AFEM_BATCH_GRAPH the zero, cell and scale passes are captured once into a
 * CUDA graph on a private stream and replayed on `stream`; the per-instance
 * table (pointers, fields) lives in device memory and is re-uploaded when
 * an argument changes, so new buffers or fields need no new capture.
 * Ownership: the batch holds the mesh handles (which must outlive it) and
 * its own device table; x_i, y_i are caller-owned device buffers,
 * x_i != y_i.  E: host [count][3] or NULL (0 field); x, y, n_vec: host
 * arrays of count entries.  Errors: AFEM_EINVAL (count outside 1..256,
 * host-only mesh or mesh on another device, n_vec_i < 1, aliased buffers),
 * AFEM_ENOMEM, AFEM_ECUDA.  Asynchronous on
 * `stream`, except that a changed table or a new signature synchronises it. */
#define AFEM_BATCH_MAX 256
#define AFEM_BATCH_GRAPH 1
#define AFEM_BATCH_MAX_CAND 8
typedef struct afem_batch afem_batch;   /* opaque */
typedef struct {
    int32_t tuned, block, grid, blocks_per_sm, n_candidates, count;
    int64_t total_cells;
    double cand_ms[AFEM_BATCH_MAX_CAND];   /* best-of-3 time of each candidate, ms */
    int32_t cand_block[AFEM_BATCH_MAX_CAND];
    int32_t cand_grid[AFEM_BATCH_MAX_CAND];
} afem_batch_tuning;
int afem_batch_create(afem_mesh* const* meshes, int count, afem_batch** out);
int afem_batch_destroy(afem_batch* batch);
int afem_batch_op_apply(afem_batch* batch, int kind, const double* E, void* const* x, void* const* y,
                        const int* n_vec, int flags, void* stream);
int afem_batch_get_tuning(const afem_batch* batch, afem_batch_tuning* out);

#ifdef __cplusplus
}
#endif
#endif /* AFEM_MCTDHF_H */
