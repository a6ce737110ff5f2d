/*
 * liblrcc: k-point-blocked LR-CCSD Jacobian products and dipole polarizability
 * for 1D periodic systems, GB300 (sm_103a).
 *
 * The method is the periodic linear-response CCSD of arXiv 2508.01266 (Caricato,
 * Parsons, Frisch, Abdoullaeva): ground-state amplitudes T and multipliers Lambda
 * plus crystal-orbital integrals in, alpha_XY(w) for chosen dipole components and
 * frequencies out (Sec. II, Eqs. 4, 12-15).
 *
 * Conventions shared by every entry point
 *   - Complex numbers are interleaved (re, im) IEEE double pairs ("c128").
 *   - Momentum: k indices 0..nk-1 on any of the meshes of Sec. II.A; conservation is
 *     k_a + k_b = k_i + k_j (mod nk) in index space (Eq. 5).
 *   - Orbitals per cell: nocc occupied then nvir virtual (n = nocc + nvir), closed
 *     shell, spatial orbitals.  Amplitudes are the alpha / alpha-beta blocks of the
 *     paper's spin-orbital amplitudes (Sec. II.A keeps all spin blocks).
 *   - Density-fitting factors L[k1][k2][Q][p][q] (paper units):
 *         <pq|rs> = (pr|qs) = sum_Q L[kp][kr][Q][p][r] * L[kq][ks][Q][q][s].
 *     Hermiticity L[k2][k1][Q] = L[k1][k2][Q]^H is required (set_integrals rejects
 *     factors that violate it beyond 1e-10 of their largest entry); it makes the
 *     paper's assumption <PQ|RS>* = <RS|PQ> (Sec. II.C) exact.
 *   - Singles x1[k][i][a]; doubles x2[ki][kj][ka][i][j][a][b] with kb implied,
 *     in the paper's normalization (t2 and lambda2 carry the factor Nk relative to
 *     the supercell amplitudes, so Eqs. 6-15 hold with their printed 1/Nk factors).
 *     Doubles must be pair-symmetric: x2[ki,kj,ka,i,j,a,b] = x2[kj,ki,kb,j,i,b,a].
 *   - The caller owns every buffer.  set_* calls copy their inputs; no pointer is
 *     retained after a call returns.  No C++ exception crosses this interface.
 *   - One problem per host thread at a time.  Device work is issued on the CUDA
 *     stream given (NULL = legacy default stream).
 */
#ifndef LRCC_H_
#define LRCC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LRCC_OK = 0,
  LRCC_EINVAL = 1,       /* bad argument, shape or state */
  LRCC_ENOMEM = 2,       /* host or device allocation failed */
  LRCC_ECUDA = 3,        /* a CUDA runtime call failed (see lrcc_last_error) */
  LRCC_ENOCONV = 4,      /* iterative solver did not reach the tolerance */
  LRCC_ETIMEOUT = 5,     /* a bounded device wait gave up */
  LRCC_EUNSUPPORTED = 6  /* option or size not supported by this build */
} lrcc_status;

typedef struct lrcc_problem lrcc_problem;
typedef struct lrcc_plan lrcc_plan;

typedef struct {
  int32_t nk, nocc, nvir, naux;
  int32_t kmesh; /* 0 Gamma-centred, 1 NRecip odd (Gamma + edge), 2 NRecip even (shifted); labels only */
} lrcc_dims;

typedef struct {
  double conv_tol;     /* convergence threshold (default 1e-10): response and Lambda equations:
                          max |residual| / max |right-hand side|; CCSD amplitudes: max |Omega|;
                          Davidson: residual norm of every wanted root */
  double refine_tol;   /* mixed precision: FP64 residual target of iterative refinement */
  int32_t max_iter;    /* default 200 */
  int32_t diis_depth;  /* default 8 */
  int32_t diis_period; /* extrapolate every n iterations (default 1) */
  int32_t precision;   /* 0 FP64, 1 TF32, 2 BF16x3 (split bf16, FP32 accumulate) */
  int32_t autotune;    /* 1: time the candidate GEMM tilings of each op once per problem and keep the fastest */
  int32_t use_graphs;  /* 1: replay each product (per direction, batch size, precision) as a CUDA graph;
                          the first call per key runs eagerly and captures the graph */
  uint64_t spin_timeout_cycles;
  int32_t response_form; /* lrcc_polarizability: 0 symmetric form (default); 1 asymmetric
                            (left-response) form, symmetrised (alpha_XY + alpha_YX) / 2;
                            2 asymmetric form as computed */
  const char* log_path;  /* NULL (default) or a file the iterative solvers append one JSON line
                            per iteration to: solver, iteration, residuals per system */
  int32_t max_batch;     /* vectors per launch of a product: 0 (default) as many as the per-vector
                            scratch that fits in device memory allows; larger batches run in
                            chunks (same results) */
  int32_t host_history;  /* DIIS history of the solvers: 0 (default) device memory unless it would
                            take more than half of the free memory, then pinned host memory read
                            by the kernels through the coherent CPU-GPU link; 1 host; -1 device */
} lrcc_options;

/* ---------------------------------------------------------------------------
 * Problem lifecycle
 * ------------------------------------------------------------------------- */

/* Create a problem for the given sizes (Sec. II.A).  *out receives a handle that
 * must be released with lrcc_destroy.  Errors: EINVAL for non-positive sizes. */
lrcc_status lrcc_create(const lrcc_dims* dims, lrcc_problem** out);

/* Integrals of Sec. II.A/II.C: DF factors (c128 [nk][nk][naux][n][n], paper units),
 * orbital energies eps ([nk][n], canonical Fock diagonal, Eq. 9) and dipole
 * integrals (c128 [3][nk][n][n], k-diagonal, <p|mu_c|q>).  Pointers are host
 * memory when on_device == 0, device memory otherwise.  Copies the data.
 * LRCC_EINVAL (problem unchanged) for non-finite values, DF factors or dipoles that
 * are not Hermitian, or a reference that is not gapped (some virtual level at or
 * below some occupied level). */
lrcc_status lrcc_set_integrals(lrcc_problem* p, const void* L, const double* eps, const void* dip,
                               int32_t on_device);

/* Ground-state amplitudes T (Eqs. 7-8) and multipliers Lambda (Eqs. 10-11),
 * paper normalization, layouts above.  l1/l2 may be NULL when only Jacobian
 * products are wanted.  Builds the T-dependent intermediates on the device. */
lrcc_status lrcc_set_ground_state(lrcc_problem* p, const void* t1, const void* t2, const void* l1,
                                  const void* l2, int32_t on_device);

/* Jacobian product on nrhs vectors (device pointers, RHS-major, each vector laid
 * out as above).  transpose == 0:  y = A x, the derivative of the CCSD residual
 * along x (the left-hand side of Eqs. 13-14, i.e. -D t plus all J terms);
 * transpose == 1:  y = P_sym A^T x under the plain array pairing
 * sum x1 y1 + sum x2 y2 (the Lambda-type product of Eqs. 10-11), P_sym = pair
 * symmetrization.  x and y must not overlap.  opt->precision selects the GEMM
 * arithmetic: 0 FP64; 1 TF32 and 2 BF16x3 (operands split in bf16 hi + lo, three
 * products) on the tcgen05 tensor cores with FP32 accumulation (data stay FP64 in
 * memory).  Asynchronous on `stream` for precision 0; the tensor-core modes
 * synchronize the stream once at the end to read the kernels' error flag
 * (LRCC_ETIMEOUT if a bounded wait gave up). */
lrcc_status lrcc_jacobian_apply(lrcc_problem* p, int32_t transpose, int32_t nrhs, const void* x1,
                                const void* x2, void* y1, void* y2, const lrcc_options* opt,
                                void* stream);

/* Same product as lrcc_jacobian_apply for one vector (nrhs = 1), for callers that
 * cannot let a library allocate device memory at call time (host applications that
 * own the device allocator, latency-critical loops that cannot absorb cudaMalloc's
 * implicit synchronization).  The paper has no counterpart; this is a property of
 * the library.  The staging vectors and the per-vector scratch live in one static
 * device array of 4 Mi complex128 elements (64 MiB) that every GPU loading the
 * library keeps until exit; the problem's own buffers (allocated by lrcc_create and
 * lrcc_set_ground_state) are used as they are.  Calls no cudaMalloc, cudaFree or
 * other allocating routine.  Problems whose vectors plus scratch exceed the array
 * return LRCC_EUNSUPPORTED with the sizes in lrcc_last_error.  The device the problem
 * was created on must be current (LRCC_EINVAL otherwise).  The first call on a device
 * (and the first after that device's context was replaced, e.g. by cudaDeviceReset)
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  Every call, from any
 * problem, shares the one array: calls whose GPU work overlaps in time race and give
 * wrong results, so serialize them (for example on one stream).  Asynchronous on
 * `stream`; x and y are device pointers laid out as for lrcc_jacobian_apply. */
lrcc_status lrcc_jacobian_apply_noalloc(lrcc_problem* p, int32_t transpose, const void* x1, const void* x2,
                                        void* y1, void* y2, void* stream);

/* Polarizability alpha_XY(w) per cell (Eq. 15), a.u., for the dipole components
 * comps[0..ncomp) (0 = x, 1 = y, 2 = z) and frequencies omegas[0..nomega).
 * opt->response_form 0: the symmetric CC linear-response function
 *   <<X;Y>>_w = 1/2 C^{+-w} [eta^X t^Y(w) + eta^Y t^X(-w) + F t^X(-w) t^Y(w)];
 * 1 and 2: the asymmetric form 1/2 C^{+-w} [eta^Y t^X(-w) + tbar^X(-w) xi^Y] with the
 * left perturbed multipliers tbar^X(w) (A + w) = -(eta^X + F t^X(w)), solved with
 * transposed Jacobian products (equal to form 0 at convergence).  alpha receives c128 [nomega][ncomp][ncomp] in host memory.
 * info (may be NULL) receives int32 [2 + ncomp]: total iterations, status of the
 * last solve, and per component 1 if it was skipped because its integrals vanish
 * (max |mu| < 1e-14, Sec. II.C).  Requires set_integrals and set_ground_state
 * with Lambda.  Synchronous. */
lrcc_status lrcc_polarizability(lrcc_problem* p, const int32_t* comps, int32_t ncomp, const double* omegas,
                                int32_t nomega, const lrcc_options* opt, void* alpha, int32_t* info);

/* Both forms of the polarizability of lrcc_polarizability from one set of right-hand
 * solutions: alpha_sym receives the symmetric form (response_form 0) and alpha_asym the
 * asymmetric (left-response) form as computed (response_form 2), each c128
 * [nomega][ncomp][ncomp] in host memory; they agree at convergence (Eq. 15 read through
 * the paper's linear-response reference), so their difference measures the solution
 * error.  opt->response_form is ignored; everything else as for lrcc_polarizability. */
lrcc_status lrcc_polarizability_forms(lrcc_problem* p, const int32_t* comps, int32_t ncomp, const double* omegas,
                                      int32_t nomega, const lrcc_options* opt, void* alpha_sym, void* alpha_asym,
                                      int32_t* info);

/* Linear-response function <<X;Y>>_w per cell (Eq. 15's response function, of which the
 * polarizability is alpha_XY = -<<mu_X;mu_Y>>) for arbitrary one-body operators instead of
 * the dipole components: electric dipole, quadrupole or magnetic-dipole-like operators, in
 * any mix.  The paper computes dipole polarizabilities and names other response
 * properties as future work (Sec. IV); the response function is the same for any
 * Hermitian one-body perturbation h -> h + eps X (Eq. 12 with X in place of mu).
 * ops: host c128 [nops][nk][n][n], <p|X_c|q> in the crystal-orbital basis, k-diagonal and
 * Hermitian per k (LRCC_EINVAL otherwise, or for non-finite elements); 1 <= nops <= 16.
 * out: host c128 [nomega][nops][nops], out[w][x][y] = <<X_x;X_y>>_w.  opt->response_form
 * and the other options as for lrcc_polarizability; info int32 [2 + nops] likewise.
 * Requires set_integrals and set_ground_state with Lambda.  Synchronous. */
lrcc_status lrcc_response_function(lrcc_problem* p, int32_t nops, const void* ops, const double* omegas,
                                   int32_t nomega, const lrcc_options* opt, void* out, int32_t* info);

/* CCSD residual Omega(t) (Eqs. 7-8, paper units, layouts as for set_ground_state) for the
 * amplitudes t1, t2 (device pointers), into r1, r2 (device).  Evaluated from Jacobian
 * products: Omega(t) = Omega(0) + 1/2 [A(s1 t) t + A(s2 t) t], s1,2 = (1 -+ 1/sqrt 3)/2,
 * exact because Omega is a polynomial of degree 4.  Requires set_integrals; the
 * problem's ground state (if set) is restored afterwards.  Synchronous. */
lrcc_status lrcc_residual(lrcc_problem* p, const void* t1, const void* t2, void* r1, void* r2);

/* Ground state on the GPU: CCSD amplitudes (Eqs. 7-8, max |Omega| <= opt->conv_tol for the
 * FP64 residual above) and the Lambda multipliers of Eqs. 10-11 (transpose products).
 * opt->precision 0: Jacobi + DIIS on the FP64 residual, Lambda in FP64 to a relative
 * residual <= opt->conv_tol.  1 (TF32) and 2 (BF16x3): inexact Newton steps for the
 * amplitudes (FP64 residual, correction A d = -Omega solved with tensor-core products to
 * 1e-4 relative for BF16x3, 3e-3 for TF32) and Lambda by iterative refinement to an FP64
 * relative residual <= opt->refine_tol.  On success they become
 * the problem's ground state (as set_ground_state with Lambda) and are also copied to
 * t1, t2, l1, l2 (each may be NULL; device memory when on_device, else host) in the
 * paper's normalization.  energy (may be NULL): CCSD correlation energy per cell.
 * info (may be NULL): int32 [4] = CCSD iterations, CCSD status, Lambda iterations,
 * Lambda status.  Requires set_integrals.  Synchronous. */
lrcc_status lrcc_solve_ground_state(lrcc_problem* p, const lrcc_options* opt, void* t1, void* t2, void* l1,
                                    void* l2, int32_t on_device, double* energy, int32_t* info);

/* Linear-response excitation energies (the poles of the response function, Eq. 15):
 * the nroots eigenvalues of the Jacobian with the smallest real parts, by a non-Hermitian
 * Davidson iteration on batched Jacobian products (orbital-energy denominator
 * preconditioner; converged when every wanted residual norm <= opt->conv_tol; products
 * in opt->precision).  omegas: host c128 [nroots].  x1, x2 (each may be NULL): device
 * c128 [nroots][Nk][o][v] and [nroots][Nk][Nk][Nk][o][o][v][v] right eigenvectors in
 * paper units, unit Hermitian norm.  info (may be NULL): int32 [2] = iterations,
 * status.  Requires set_ground_state; 1 <= nroots <= Nk o v.  Synchronous. */
lrcc_status lrcc_excitation_energies(lrcc_problem* p, int32_t nroots, const lrcc_options* opt, void* omegas,
                                     void* x1, void* x2, int32_t* info);

/* Polarizabilities of several independent problems (for example chains of different
 * Nk, o, v) in one call, all with the same components, frequencies and options.  Each
 * problem's solve runs on its own host thread and that thread's default stream, so
 * the problems' kernels share the GPU.  alphas[i] and infos[i] are as for
 * lrcc_polarizability (infos, or any entry of it, may be NULL).  The problems must be
 * distinct handles on the calling thread's current device.  Every problem is
 * attempted; returns the first non-OK status in problem order.  Synchronous. */
lrcc_status lrcc_batch_polarizability(lrcc_problem* const* probs, int32_t nprob, const int32_t* comps,
                                      int32_t ncomp, const double* omegas, int32_t nomega,
                                      const lrcc_options* opt, void* const* alphas, int32_t* const* infos);

/* Last error message of a problem (static storage owned by the handle). */
const char* lrcc_last_error(const lrcc_problem* p);

/* Release every host and device resource of a problem.  NULL is ignored. */
void lrcc_destroy(lrcc_problem* p);

/* Default options. */
void lrcc_default_options(lrcc_options* opt);

/* Number of device kernels this problem has launched so far (a counter kept by
 * the executor; -1 for a NULL handle). */
int64_t lrcc_kernel_launches(const lrcc_problem* p);

/* Per-op timing: when enabled, every op the executor launches is bracketed by CUDA
 * events recorded on its launching stream (cleared on each call to this function).
 * lrcc_profile_query sums, over the recorded ops whose tag equals `tag` (an empty
 * string selects all), the event-timed milliseconds, the launch count and the
 * algorithmic real flops (8 per complex multiply-add).  Query synchronizes the
 * device.  Tags are the op names of the plan (e.g. "ladder", "W build"). */
lrcc_status lrcc_profile(lrcc_problem* p, int32_t enable);
lrcc_status lrcc_profile_query(lrcc_problem* p, const char* tag, double* ms, int64_t* count, double* flops);
/* All recorded ops aggregated by tag, slowest first: one line per tag,
 * "tag<TAB>ms<TAB>count<TAB>flops<LF>", NUL-terminated in buf[len].  Returns
 * LRCC_EINVAL (with the report truncated) when len is too small. */
lrcc_status lrcc_profile_report(lrcc_problem* p, char* buf, int64_t len);

/* ---------------------------------------------------------------------------
 * Plan introspection (host only; never touches the GPU)
 *
 * The Jacobian is executed as a fixed list of ops: segmented batched complex
 * GEMMs, momentum-aware layout permutations and batched 2-D transposes over five
 * arenas (0 fixed data, 1 input vector, 2 output vector, 3 per-vector scratch,
 * 4 W-block workspace).  These calls expose that list so its index arithmetic can
 * be checked on a CPU.  which: 0 ground-state program, 1 Jacobian, 2 transposed
 * Jacobian, 3 perturbation right-hand side (Eq. 12), 4 energy second derivative,
 * 5 residual at zero amplitudes, 6 energy gradient with respect to the amplitudes.
 * ------------------------------------------------------------------------- */
lrcc_status lrcc_plan_create(const lrcc_dims* dims, int64_t ws_budget, lrcc_plan** out);
void lrcc_plan_destroy(lrcc_plan* h);
/* arena_sizes int64[5] (complex elements); offsets int64[11]: Loo, Lov, Lvo, Lvv,
 * f0, t1, t2, identity, x1, x2, one-body operator blocks; flops double[3]:
 * Jacobian, ladder, W build. */
lrcc_status lrcc_plan_info(const lrcc_plan* h, int64_t* arena_sizes, int64_t* offsets, double* flops);
int32_t lrcc_plan_num_ops(const lrcc_plan* h, int32_t which);
/* Bounds check of every op of every program against the arena sizes; writes a
 * NUL-terminated message (empty when every access is in bounds) into msg[len]. */
lrcc_status lrcc_plan_validate(const lrcc_plan* h, char* msg, int32_t len);
/* kind_idx_fixed int32[3]: kind (0 GEMM, 1 permute, 2 2-D transpose, 3 zero a
 * scratch range), table index, fixed-only flag. */
lrcc_status lrcc_plan_op(const lrcc_plan* h, int32_t which, int32_t i, int32_t* kind_idx_fixed);
/* ints int32[16]: M N K ta tb arA arB arC epi ep0..ep3 nbatch nseg store; lds int64[3];
 * alpha double[2]; coff int64[nbatch], sbeg int32[nbatch+1], aoff/boff int64[nseg].
 * store = 1: C = alpha * sum instead of C += alpha * sum (the GEMM is the first writer of a
 * scratch buffer and covers all of it, in place of zeroing the buffer first). */
lrcc_status lrcc_plan_gemm(const lrcc_plan* h, int32_t idx, int32_t* ints, int64_t* lds, double* alpha,
                           int64_t* coff, int32_t* sbeg, int64_t* aoff, int64_t* boff);
/* Kernel the executor launches by default for GEMM op idx at a precision (0 FP64,
 * 1 TF32, 2 BF16x3), as decided on the host before any launch; out int32[7]: packed
 * (tensor-core kernel on packed operands), special (1 short-contraction, 2 tiny-output
 * reduction kernel), tc (unpacked tensor-core kernel), f32 (FP32 arithmetic on FP64
 * operands), tile (tiled-kernel shape), nsplit (K splits; the reduction kernel splits
 * whole segments), max_seg (most segments of a batch entry).  The mixed-precision modes are
 * this library's (the paper computes in FP64); they keep every FP32 accumulation chain
 * within 8192 complex terms, the partials of K splits being summed in FP64.  EINVAL for a
 * bad handle, index or precision. */
lrcc_status lrcc_plan_choice(const lrcc_plan* h, int32_t idx, int32_t precision, int32_t* out);
/* ints int32[19]: src(kind nk n0..n3) dst(kind nk n0..n3) pi0..pi3 arS arD store; offs int64[2].
 * store = 1: the permutation overwrites its destination (dst = alpha * src) instead of adding
 * to it; the plan sets it where the permutation is the first writer of a scratch buffer and
 * covers all of it, in place of zeroing the buffer first. */
lrcc_status lrcc_plan_perm(const lrcc_plan* h, int32_t idx, int32_t* ints, int64_t* offs, double* alpha);
/* ints int32[5]: nb R C arS arD; offs int64[2]. */
lrcc_status lrcc_plan_btrans(const lrcc_plan* h, int32_t idx, int32_t* ints, int64_t* offs, double* alpha);
/* Zero op: arena, first element and element count of the range set to zero in every
 * right-hand side's copy of the arena.  Scratch buffers whose lifetimes do not overlap
 * share memory; each starts its lifetime with such an op. */
lrcc_status lrcc_plan_zero(const lrcc_plan* h, int32_t idx, int32_t* arena, int64_t* off_n);

/* Self test of the bounded device waits: launches one thread that waits on an mbarrier
 * nothing arrives at, for at most `polls` polls, then records the timeout in the
 * problem's device error flag (the mechanism every tensor-core kernel uses when a copy
 * or an MMA never completes).  Returns LRCC_ETIMEOUT after reading and clearing the flag;
 * the context stays usable.  Synchronous. */
lrcc_status lrcc_wait_selftest(lrcc_problem* p, int64_t polls);

/* Host-only utility: eigenvalues w (c128 [n]) and unit right eigenvectors v (c128
 * [n][n], row-major, columns are the vectors; may be NULL) of the row-major complex
 * n x n matrix a (Hessenberg reduction and shifted QR).  It solves the Davidson subspace
 * problem of lrcc_excitation_energies and is exported for tests.  LRCC_ENOCONV if the
 * iteration fails. */
lrcc_status lrcc_small_eig(int32_t n, const void* a, void* w, void* v);

#ifdef __cplusplus
}
#endif

#endif /* LRCC_H_ */
