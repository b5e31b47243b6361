/*
 * dwsolve.h -- C ABI of the GB300 deflated SAP-GCR solver for the
 * O(a)-improved Wilson-Dirac equation  D psi = eta  (paper eq. (3.9)).
 *
 * Method: M. Luescher, "Local coherence and deflation of the low quark
 * modes in lattice QCD" (Sections 3-6 and Appendix A).
 *
 * Conventions shared by every call
 * --------------------------------
 *  Lattice L[0] x L[1] x L[2] x L[3], L[0] = time.  Canonical site index
 *  ((x0*L1 + x1)*L2 + x2)*L3 + x3 (x0 slowest), V = L0*L1*L2*L3.
 *  Canonical quark field: V x 4 (spin) x 3 (colour) complex numbers, each
 *  complex stored as two doubles (re, im) -- "complex128[V][4][3]".
 *  Canonical gauge field: V x 4 (mu) x 3 x 3 complex, U[x][mu] = link from
 *  x to x+mu, row-major colour matrix.  Links must be SU(3) (unitary,
 *  det 1): the library stores two rows and rebuilds the third.
 *
 *  D psi(x) = (4+m0) psi(x) + c_sw (i/4) sum_{mu,nu} sigma_{mu nu} F_{mu nu}(x) psi(x)
 *             - 1/2 sum_mu [(1-gamma_mu) U_mu(x) psi(x+mu) + (1+gamma_mu) U_mu(x-mu)^+ psi(x-mu)]
 *  in the Euclidean chiral basis (gamma_0 = [[0,-1],[-1,0]],
 *  gamma_k = [[0,-i s_k],[i s_k,0]], gamma_5 = diag(1,1,-1,-1)), clover-leaf
 *  F_{mu nu}, fermion field antiperiodic in time when requested.
 *
 *  "Packed" fields are the library's internal device layout (block-major
 *  site order, structure of arrays).  Convert with dw_pack / dw_unpack;
 *  dw_field_bytes gives the size of one packed field.  Packed fields of
 *  precision DW_F64 hold doubles, DW_F32 floats.
 *
 *  Memory: every *_dev pointer is device memory owned by the caller; the
 *  library never frees it.  Contexts own their internal buffers and free
 *  them in *_destroy.  Streams: `stream` is a cudaStream_t (NULL = legacy
 *  default stream); calls are stream-ordered unless documented as
 *  synchronous.  One context must not be used by two host threads at once.
 *  A context belongs to the device that was current at dw_create; calls that
 *  take it (dw_apply, dw_apply_schur_static, sap_precondition, deflation_build,
 *  gcr_solve, cgnr_solve) return DW_EINVAL when another device is current.
 *
 *  Errors: functions return a dw_status.  Negative values are failures
 *  (nothing useful was written); positive values are successes with a
 *  caveat.  No exceptions cross the ABI.
 */
#ifndef DWSOLVE_H
#define DWSOLVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DW_OK = 0,
  DW_EINVAL = -1,      /* invalid argument, lattice/block mismatch, non-SU(3) links, rank loss */
  DW_ENOMEM = -2,      /* device allocation failed */
  DW_ECUDA = -3,       /* a CUDA call failed (message via dw_last_error) */
  DW_ENOTCONV = 1,     /* iteration limit reached before the tolerance */
  DW_ILLCOND = 2       /* a diagonal little block was ill-conditioned (Appendix A.2) */
} dw_status;

/* DW_F64X: FP64 fields and results, computed in double-float arithmetic (each real as the
 * unevaluated sum of two FP32 values, about 48 significant bits) on the FP32 pipes, whose rate on
 * this GPU is many times its FP64 rate; accepted by dw_apply (DW_OP_FULL), dfl_restrict and
 * dfl_prolong, and used for the restart steps of the mixed-precision solver.  Relative error of
 * D in a few 1e-14. */
typedef enum { DW_F64 = 0, DW_F32 = 1, DW_BF16 = 2, DW_F64X = 3 } dw_prec;

typedef enum { DW_OP_FULL = 0, DW_OP_SCHUR = 1 } dw_op;

typedef struct dw_ctx dw_ctx;
typedef struct dfl_ctx dfl_ctx;

typedef struct {
  int L[4];            /* lattice extents, L[0] = time; each a multiple of sap_bs[mu] */
  double m0;           /* bare mass; hopping parameter kappa = 1/(2 m0 + 8) */
  double csw;          /* Sheikholeslami-Wohlert coefficient */
  int antiperiodic;    /* 1: antiperiodic fermion boundary in time, 0: periodic */
  int sap_bs[4];       /* Schwarz block size: even extents, even block count per direction, <= 512 sites */
} dw_params;

/* Last error message of the calling thread (static storage, never NULL). */
const char* dw_last_error(void);
/* Number of CUDA kernels this library has launched in the process so far
 * (all contexts); callers difference two readings to count the launches of
 * a region. */
long long dw_launch_count(void);

/* Create an operator context from host links (canonical layout, FP64).
 * Builds the clover term F, A(x) = (4+m0) + c_sw (i/4) sigma F and its
 * inverse per chiral 6x6 block in FP64 (Section 2.1 operator), and FP32
 * copies.  Synchronous.  Returns DW_EINVAL on bad extents or non-SU(3)
 * links (|U U^+ - 1| or |det U - 1| above 1e-10). */
int dw_create(const dw_params* p, const double* links_host, dw_ctx** out);
void dw_destroy(dw_ctx* ctx);

/* Free the workspaces a context keeps between calls (solver Krylov fields, the double-float copies
 * of links and clover term); later calls allocate them again.  Synchronises the device. */
int dw_release_workspace(dw_ctx* ctx);

/* Bytes of one packed field of precision prec (DW_F64 or DW_F32). */
size_t dw_field_bytes(const dw_ctx* ctx, int prec);
/* Number of lattice sites V. */
long long dw_volume(const dw_ctx* ctx);

/* canonical complex128[nrhs][V][4][3] (device)  <->  nrhs packed fields (device). */
int dw_pack(dw_ctx* ctx, int prec, int nrhs, const double* canon_dev, void* packed_dev, void* stream);
int dw_unpack(dw_ctx* ctx, int prec, int nrhs, const void* packed_dev, double* canon_dev, void* stream);

/* out = D in (op = DW_OP_FULL) or, on even sites, out = (A_ee - D_eo A_oo^{-1} D_oe) in
 * with odd sites of out set to zero (op = DW_OP_SCHUR; even-odd Schur complement).
 * in/out: nrhs packed fields of precision prec; in != out.  prec DW_F64X: FP64 packed fields
 * (pack with DW_F64), DW_OP_FULL only, computed in double-float arithmetic. */
int dw_apply(dw_ctx* ctx, int prec, int op, int nrhs, const void* in_dev, void* out_dev, void* stream);

/* The Schur complement of dw_apply(DW_OP_SCHUR) for one field, allocating no memory.  The
 * paper has no counterpart: this is an interface for callers that must not allocate device
 * memory at the time of the call (cudaMalloc synchronises the device, stalling other
 * streams, and can fail under a fixed memory reservation), whereas dw_apply allocates its
 * intermediate field on first use.  The intermediate A_oo^{-1} D_oe in lives in a fixed
 * 16 MiB device array of the library: volumes whose packed field of precision prec exceeds
 * 16 MiB (FP64: more than 87381 sites; FP32: more than 174762) get DW_EINVAL with a message.
 * The first call on each device looks up the array's address (set-up, once per device; make
 * it before any stream capture).  The array is shared by all calls on a device: calls that
 * overlap in time (other streams, other host threads) race on it and must be ordered by the
 * caller.  in/out: one packed field of precision prec (device), in != out; odd sites of out
 * are set to zero.  Results equal those of dw_apply(DW_OP_SCHUR). */
int dw_apply_schur_static(dw_ctx* ctx, int prec, const void* in_dev, void* out_dev, void* stream);

/* xi = M_sap rho: Schwarz alternating procedure (Section 6.1) on the
 * sap_bs blocks, ncy cycles of (black blocks, white blocks), each block
 * solve = nmr minimal-residual steps on the even-odd preconditioned block
 * operator with Dirichlet block boundary.  rho, xi: packed, prec
 * DW_F32 or DW_F64; rho != xi.  Uses internal workspace of the context. */
int sap_precondition(dw_ctx* ctx, int prec, int ncy, int nmr, int nrhs,
                     const void* rho_dev, void* xi_dev, void* stream);

typedef struct {
  int bs[4];           /* deflation block size: multiple of sap_bs, even block count per direction */
  int Ns;              /* fields per block, 1..32 */
  int n_inv;           /* inverse-iteration steps (5.1); 0 = use the start fields as they are */
  int ncy, nmr;        /* M_sap parameters used by the inverse iteration */
  int basis_prec;      /* DW_BF16: BF16 basis + FP32 little operator copy (mixed path);
                          DW_F64: FP64 basis (plain path) */
  int iter_prec;       /* precision of the inverse iteration: DW_F32 or DW_F64 */
  double cond_max;     /* largest accepted condition number of a diagonal little block (A.2) */
  /* learned generation (optional; iter_prec must be DW_F32): after net_k0 plain steps the fields go
   * through the parallel-transport network (weights: ptnet_weight_count(net_channels) complex FP32),
   * unless the network output fails the judge -- mean ||D psi||/||psi|| must fall below
   * net_judge times its value at the network input -- in which case the plain steps continue. */
  const void* net_weights;   /* NULL: plain procedure only */
  int net_channels;          /* 16 */
  int net_k0;                /* plain steps before the network */
  double net_judge;          /* e.g. 0.95 */
  /* bootstrapped generation (Section 5.3): after the n_inv plain steps, boot_steps further steps
   * psi_l <- chi_l / ||chi_l|| with D chi_l = psi_l solved approximately by the mixed-precision
   * DFL+SAP+GCR solver deflated by the block subspace of the current fields (relative tolerance
   * boot_tol, at most boot_nmx GCR steps; the Ns fields as one batch).  0: plain procedure only.
   * The generation runs with the context's operator; the paper recommends a bare mass close to the
   * critical one for it -- build on such a context and move the subspace with dfl_retarget. */
  int boot_steps;
  double boot_tol;           /* e.g. 1e-2 */
  int boot_nmx;              /* e.g. 16 */
} dfl_params;

typedef struct {
  double seconds;          /* wall time of the build */
  double seconds_little;   /* of which: little operator assembly (A.1)-(A.3) */
  double max_block_cond;   /* largest condition-number estimate of B_LL */
  int Nb;                  /* number of deflation blocks */
  int N;                   /* little dimension Nb * Ns */
  int learned_used;        /* 1: the network output was accepted */
  double rho_in;           /* mean ||D psi||/||psi|| at the network input (after net_k0 steps) */
  double rho_out;          /* ... of the network output (or of the fields after the plain fallback); without a
                              network: of the generated fields (FP32 generation only, else 0) */
  int boot_steps;          /* bootstrapped steps done */
  int boot_gcr_steps;      /* GCR steps of their approximate solves, summed over steps and fields */
  int little_loaded;       /* dfl_load: 1 if the stored little operator was used (same operator) */
} dfl_info;

/* Build the deflation subspace (Sections 4.2, 5.3) and the little Dirac
 * operator (3.2), (A.1)-(A.3).  start_canon_dev: Ns random fields,
 * complex128[Ns][V][4][3] (the random numbers are an input).  Steps:
 * n_inv x (psi_l <- M_sap psi_l, normalised); block restriction and
 * Gram-Schmidt (FP64, two passes); optional BF16 rounding of the basis;
 * FP64 assembly of B_{LL'} from the stored (rounded) basis; inverses of
 * the diagonal blocks; global-mode deflation data.  Synchronous.
 * Returns DW_ILLCOND if a diagonal block exceeds cond_max (the context is
 * still created; the little solver then works on the full system). */
int deflation_build(dw_ctx* ctx, const dfl_params* p, const double* start_canon_dev,
                    dfl_ctx** out, dfl_info* info);
void dfl_destroy(dfl_ctx* d);
int dfl_dims(const dfl_ctx* d, int* Nb, int* Ns);

/* Subspace reuse (Section 6.4, remark 1: one deflation subspace serves all valence masses): a new
 * deflation context on operator ctx (same lattice and Schwarz blocks as the operator src was built
 * on; another bare mass, c_sw or gauge field) with the basis and global-mode data of src, its own
 * little operator (A.1) and A.2/A.3 data.  Synchronous; may return DW_ILLCOND like deflation_build. */
int dfl_retarget(const dfl_ctx* src, dw_ctx* ctx, dfl_ctx** out, dfl_info* info);
/* Checkpoint of a deflation subspace: lattice, block sizes, Ns, the stored basis (BF16 or FP64),
 * the global-mode restriction coefficients (A.3) and the FP64 little operator with the identity
 * of the operator it belongs to (gauge-field hash, m0, c_sw).  Binary file, host byte order.
 * dfl_load rebuilds the context on ctx: the stored little operator is used when ctx is the same
 * operator (info->little_loaded = 1), otherwise it is assembled anew.  DW_EINVAL on I/O errors or
 * a lattice/block mismatch.  Synchronous. */
int dfl_save(const dfl_ctx* d, const char* path);
int dfl_load(dw_ctx* ctx, const char* path, dfl_ctx** out, dfl_info* info);

/* Little vectors: complex[Nb][Ns] (re, im interleaved) of precision prec,
 * block index = lexicographic deflation-block coordinate (x0 slowest).
 * c = Phi^+ psi  (block restriction of (4.1));  psi = Phi c  (prolongation).
 * prec DW_F64X: FP64 fields and little vectors, computed in double-float arithmetic. */
int dfl_restrict(dfl_ctx* d, int prec, const void* psi_packed_dev, void* c_dev, void* stream);
int dfl_prolong(dfl_ctx* d, int prec, const void* c_dev, void* psi_packed_dev, void* stream);
/* The stored basis as canonical FP64 fields complex128[Ns][V][4][3]: field l
 * is sum over blocks of phi^L_l (dequantised when stored in BF16). */
int dfl_basis_export(dfl_ctx* d, double* canon_dev, void* stream);
/* w = A v with the little operator (3.2)/(A.1) (FP64 master copy). */
int little_apply(dfl_ctx* d, const double* v_dev, double* w_dev, void* stream);
/* Solve A v = w (6.1) by even-odd preconditioning (A.2), global-mode
 * deflation (A.3) and GCR (A.4) to ||w - A v|| <= tol ||w|| (measured on
 * the even-odd deflated system).  prec: DW_F32 (FP32 operator copy) or
 * DW_F64.  Synchronous with respect to the host (returns the counts). */
int little_dirac_solve(dfl_ctx* d, int prec, const void* w_dev, void* v_dev, double tol, int maxit,
                       int* iters, double* relres, void* stream);

/* nrhs little systems A v_r = w_r at once (Appendix A.2-A.4, as little_dirac_solve), w/v:
 * nrhs little vectors one after the other.  prec DW_F32: the FP32 systems run in lockstep in one
 * cooperative launch per group of up to 12 right-hand sides (each with its own scalars and
 * convergence), tol relative to each ||w_r|| on the even-odd deflated system.  prec DW_F64: FP64
 * vectors, iterative refinement (FP64 residual of the full little system, FP32 lockstep correction
 * solves) to ||w_r - A v_r|| <= tol ||w_r|| -- the restart solves of the batched mixed solver.
 * 1 <= nrhs <= 64.  iters/relres: nrhs entries (may be NULL).  Returns DW_ENOTCONV when a system
 * missed the tolerance.  Synchronous. */
int little_dirac_solve_batch(dfl_ctx* d, int prec, int nrhs, const void* w_dev, void* v_dev, double tol,
                             int maxit, int* iters, double* relres, void* stream);

typedef struct {
  double tol;              /* stop when ||eta - D psi|| <= tol ||eta|| (FP64 residual) */
  int nkv;                 /* Krylov vectors per GCR cycle (restart length) */
  int nmx;                 /* maximum total GCR steps */
  int ncy, nmr;            /* M_sap parameters; ncy = 0: no preconditioner (M = 1), i.e. plain GCR */
  int mixed;               /* 1: FP32 D/SAP/little, FP64-class restarts (double-float D, restriction
                              and prolongation, FP64-refined little solves); 0: everything FP64 */
  double inner_rtol;       /* mixed: end a cycle when its residual drops by this factor */
  double little_tol_out;   /* little-solve tolerance outside cycles (A.5), e.g. 1e-12 */
  double little_tol_in;    /* inside cycles, scaled by ||rho_0|| / ||D xi_k|| (A.5), e.g. 1e-6 */
  double little_tol_cap;   /* upper limit of the adapted tolerance, e.g. 1e-1 */
  int little_nkv, little_maxit;
} sol_params;

typedef struct {
  int status;              /* dw_status of this right-hand side */
  int iterations;          /* GCR steps (Krylov vectors generated) */
  int restarts;
  int little_iterations;   /* total little GCR steps */
  int little_solves;
  double relres;           /* final ||eta - D psi|| / ||eta|| in FP64 */
  double seconds;          /* wall time */
  double t_sap, t_dirac, t_project, t_little, t_orth, t_restart;  /* phase times (s), CUDA events */
} sol_info;

/* Solve D psi = eta (3.9) for nrhs right-hand sides: FGCR (Section 6.2)
 * right-preconditioned by M_sap, deflated by d (Sections 3.2, 6.1) with
 * adapted little-solve precision (A.5); d = NULL gives SAP+GCR.
 * Mixed precision with nrhs > 1 runs the right-hand sides in lockstep (one batch through every
 * kernel, M_sap from captured CUDA graphs, the little solves of each step in one multi-RHS
 * launch of up to 12 systems); environment DW_BATCH=0 solves them one after the other.
 * eta, psi: canonical complex128[nrhs][V][4][3] on the device.
 * info: nrhs entries (may be NULL).  Synchronous. */
int gcr_solve(dw_ctx* ctx, dfl_ctx* d, const sol_params* p, int nrhs, const double* eta_dev,
              double* psi_dev, sol_info* info, void* stream);

/* Autotuner: times the candidate launch shapes of the hot kernels on this
 * context's lattice for nrhs right-hand sides (multi-RHS D: one thread per site and
 * right-hand side with the site chunks interleaved, or one thread per site with
 * 1..3 right-hand sides per pass; Schwarz kernel: staged or generic FP32 variant) with CUDA events,
 * keeps the fastest in the context and writes a JSON summary to report
 * (may be NULL).  Synchronous; allocates two temporary batches of fields. */
int dw_autotune(dw_ctx* ctx, int nrhs, char* report, size_t report_len);

/* Shape sweep of the FP32 cooperative little solver of d: grid sizes (all SMs, 3/4 and 1/2 of them)
 * x hop variant (operator staged through a shared-memory ring by bulk copies / register-pipelined
 * loads), timed with CUDA events on little solves of a fixed right-hand side; the fastest per
 * iteration is kept in d.  JSON summary in report (may be NULL).  Synchronous. */
int dfl_autotune(dfl_ctx* d, char* report, size_t report_len);

/* Parallel-transport network of the learned subspace generation (3 layers, 1 -> C -> C -> 1
 * channels; each layer h'(x) = sum over the 9 transports {1, U_mu(x) . (x+mu), U_mu(x-mu)^+ . (x-mu)}
 * of a (channel x spin) matrix; gauge covariant).  Weights: ptnet_weight_count(C) complex FP32
 * (layers back to back, each [9][4 C_out][4 C_in] row-major).  Only C = 16 is built. */
size_t ptnet_weight_count(int C);
/* y_f = N(x_f) for nf packed FP32 fields.  Synchronous. */
int ptnet_forward(dw_ctx* ctx, int C, const void* weights, int nf, const void* x, void* y, void* stream);
/* Loss L = sum_f |N(x_f) - y_f|^2 / sum_f |y_f|^2 and gradient dL/dRe W + i dL/dIm W (same layout
 * as the weights), computed by the network's backward kernels.  Synchronous. */
int ptnet_loss_grad(dw_ctx* ctx, int C, const void* weights, int nf, const void* x, const void* y, void* grad,
                    double* loss, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999) on ncomplex complex weights; m, v: optimiser state. */
int ptnet_adam(size_t ncomplex, void* weights, const void* grad, void* m, void* v, int step, double lr,
               void* stream);
/* One 16 -> 16 channel layer of the network: out = sum_d W_d T_d in, or its adjoint
 * sum_d W_d^+ T_d^+ in (adjoint = 1; the data gradient of back-propagation).  W: the layer's
 * [9][64][64] complex FP32 weights; in/out: 16 packed FP32 channel fields each (one after the other).
 * tensor_cores = 1: the 5th-generation tensor cores (tcgen05, BF16 operands, FP32 accumulation;
 * relative error a few 1e-3), 0: FP32 on the CUDA cores.  Synchronous.  DW_ECUDA if a wait on the
 * tensor core or a bulk copy timed out. */
int ptnet_layer16(dw_ctx* ctx, const void* W, int adjoint, int tensor_cores, const void* in, void* out, void* stream);
/* ptnet_forward with the 16 -> 16 layer on the tensor cores (BF16 operands, FP32 accumulation). */
int ptnet_forward_tc(dw_ctx* ctx, int C, const void* weights, int nf, const void* x, void* y, void* stream);
/* The plain subspace generation (5.1) on nf packed FP32 fields in place: nsteps times
 * psi <- M_sap psi, normalised.  Synchronous. */
int dfl_inverse_iteration(dw_ctx* ctx, int ncy, int nmr, int nsteps, int nf, void* fields, void* stream);

/* Conjugate gradient on the normal equations D^+ D psi = D^+ eta, FP64,
 * unpreconditioned (the plain iterative method against which the paper's
 * near-critical masses are characterised).  Stops at
 * ||eta - D psi|| <= tol ||eta|| or after maxit iterations (DW_ENOTCONV).
 * eta, psi: canonical complex128[V][4][3] on the device.  Synchronous. */
int cgnr_solve(dw_ctx* ctx, double tol, int maxit, const double* eta_dev, double* psi_dev, int* iters,
               double* relres, void* stream);

/* EO+BiCGstab, the first comparison solver of Table 1 (Section 6.3): BiCGstab on the even-odd
 * preconditioned operator A_ee - D_eo A_oo^{-1} D_oe (the DW_OP_SCHUR operator), FP64, with the
 * odd part reconstructed exactly.  Stops at ||eta - D psi|| <= tol ||eta|| (checked with D) or
 * after maxit iterations (DW_ENOTCONV); iters counts BiCGstab iterations (two even-odd operator
 * applications each).  eta, psi: canonical complex128[V][4][3] on the device.  Synchronous. */
int bicgstab_solve(dw_ctx* ctx, double tol, int maxit, const double* eta_dev, double* psi_dev, int* iters,
                   double* relres, void* stream);

/* The nev lowest eigenvalues and eigenvectors of D^+ D by Chebyshev-accelerated subspace iteration,
 * the method the paper uses for all its eigenmode computations (Section 2.2): a block of nev + nbuf
 * fields (start: canonical complex128[nev+nbuf][V][4][3], random numbers given by the caller) is
 * filtered by the Chebyshev polynomial of degree `degree` on [a, b] (a: largest Ritz value of the
 * block, b: 1.1 x a power-iteration estimate of the largest eigenvalue), re-orthonormalised and
 * Rayleigh-Ritz projected (FP64) until ||D^+D x_i - theta_i x_i|| <= tol theta_i for the nev lowest
 * or maxit iterations (DW_ENOTCONV).  prec: precision of the filter (DW_F32 or DW_F64).
 * modes: canonical complex128[nev][V][4][3] (orthonormal), evals / resid: nev doubles (resid may be
 * NULL).  nev + nbuf <= 128.  Synchronous; the workspace (3 FP64 and 3 prec blocks of nev + nbuf
 * fields) is kept by the context. */
int lowmodes_solve(dw_ctx* ctx, int nev, int nbuf, int degree, double tol, int maxit, int prec,
                   const double* start_dev, double* modes_dev, double* evals, double* resid, int* iters,
                   void* stream);
/* Deficits (3.15) eps_f = ||(1 - P) psi_f||^2 / ||psi_f||^2 of nf fields (canonical
 * complex128[nf][V][4][3], device) with respect to the block subspace of d (projector (4.1), FP64
 * arithmetic on the stored basis) -- the local-coherence measurement of Section 5.2.  eps: nf
 * doubles (host).  Synchronous. */
int dfl_deficits(dfl_ctx* d, int nf, const double* fields_dev, double* eps, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DWSOLVE_H */
