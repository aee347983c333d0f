/*
 * helm.h -- C ABI of libhelm: the diagonal sweeping source-transfer domain
 * decomposition method for the Helmholtz equation (Leng & Ju, "A diagonal
 * sweeping domain decomposition method with source transfer for the Helmholtz
 * equation"), on one GB300 GPU (sm_103a).
 *
 * Problem (Section 1, Eq. 1.1):  Delta u + kappa^2 u = f  in R^n, n = 2, 3,
 * kappa = omega / c(x), Sommerfeld radiation condition (Eq. 1.2), truncated by
 * a uniaxial PML (Section 2.1, Eq. 2.1-2.2) with alpha_j = 1 + i sigma_j and
 * sigma(t) = sigma0 (t/L)^power, discretised by second-order central
 * differences (5-point in 2D, 7-point in 3D; Section 5) in the J-multiplied
 * form  div(A grad u) + J kappa^2 u = J f.
 *
 * Grid conventions (all arrays):
 *   - The full grid is the interior, n[a] cells per axis, plus pml.width cells
 *     on every side: N[a] = n[a] + 2*width.  Nodes are cell centred.
 *   - Arrays over it are row-major with x fastest: index ((z*Ny)+y)*Nx + x.
 *   - Complex arrays are interleaved complex128 (re, im), laid out
 *     [rhs][full grid].  Real arrays are float64.
 *
 * Memory: every entry point that takes data pointers also takes `mem`:
 * HELM_MEM_HOST (pageable or pinned host memory; the library copies in and
 * out, synchronously, through up to three device staging buffers that the
 * context keeps between calls -- they only grow, and helm_destroy frees them)
 * or HELM_MEM_DEVICE (CUDA device pointers valid in the
 * current device's primary context; work is queued on the context's stream
 * and completed before return).  The caller owns every pointer it passes; the
 * library copies what it needs and never keeps a caller pointer.
 *
 * Errors: every int-returning call returns HELM_OK (0) or a negative code.
 * On error the context stays usable unless the code is HELM_ERR_CUDA.
 * helm_strerror() names a code; helm_last_error() gives the last message of
 * the calling thread.
 *
 * Threads and streams: one context must not be used by two host threads at
 * once.  All device work of a context runs on its stream (helm_config.stream
 * or a stream the library creates).
 */
#ifndef HELM_H
#define HELM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum helm_status {
    HELM_OK = 0,
    HELM_ERR_ARG = -1,            /* invalid argument or unsupported size */
    HELM_ERR_OOM = -2,            /* device allocation failed */
    HELM_ERR_NOT_FACTORED = -3,   /* solve before helm_factor */
    HELM_ERR_NO_CONVERGENCE = -4, /* GMRES hit maxit; output and stats still written */
    HELM_ERR_TIMEOUT = -5,        /* a bounded device wait expired */
    HELM_ERR_CUDA = -6,           /* a CUDA runtime call failed */
    HELM_ERR_NUMERIC = -7         /* NaN/Inf or zero pivot in a factor */
};

enum helm_precision {
    HELM_PREC_F64 = 0,   /* complex128 factors and local solves (plain FP64 DDM) */
    HELM_PREC_MIXED = 1, /* complex64 factors and local solves, FP64 outer GMRES */
    HELM_PREC_TF32 = 2,  /* complex64 factors, local block products on the tensor
                            cores in TF32 with FP32 accumulation, FP64 outer GMRES */
    HELM_PREC_F16 = 3    /* as HELM_PREC_TF32, but where the two-ended tensor-core solve
                            applies its operands are FP16 (the same 10-bit mantissa as
                            TF32) with power-of-two scales per factor line and per
                            right-hand-side column, half the bytes and MMAs */
};

enum helm_pml_form {
    HELM_PML_LITERAL = 0, /* alpha = 1 + i sigma          (Eq. 2.1 as printed) */
    HELM_PML_OMEGA = 1    /* alpha = 1 + i sigma / omega  (frequency-scaled)  */
};

enum helm_mem { HELM_MEM_HOST = 0, HELM_MEM_DEVICE = 1 };

typedef struct helm_ctx helm_ctx;

/* Global PML (Section 2.1, Eq. 2.1): `width` cells on each side of the
 * interior, sigma(t) = sigma0 (t / (width*h))^power at distance t into it. */
typedef struct {
    int32_t width;
    int32_t power;
    double sigma0;
    int32_t form; /* enum helm_pml_form */
} helm_pml;

/* Checkerboard partition (Section 2.1): nb[a] boxes per axis.  cuts[a], if
 * not NULL, holds nb[a]+1 increasing box faces in interior cells with
 * cuts[a][0] = 0 and cuts[a][nb[a]] = n[a]; NULL means uniform boxes.  Edge
 * boxes extend over the global PML.  Each subdomain problem P_{Omega_ij} has
 * `overlap` (d) cells of zero sigma beyond an internal box face followed by
 * `sub_pml` PML cells (shifted profile, Eq. 2.3); sub_pml = 0 means
 * pml.width.  Every box must be at least overlap + 2 cells wide (in 3D an
 * inner box at least 2 overlap) and every window must stay inside the full
 * grid; helm_setup returns HELM_ERR_ARG otherwise. */
typedef struct {
    int32_t nb[3];
    const int64_t *cuts[3];
    int32_t overlap;
    int32_t sub_pml;
} helm_partition;

/* Implementation knobs.  Zero-initialise for defaults. */
typedef struct {
    int32_t precision;  /* enum helm_precision (default HELM_PREC_MIXED) */
    int32_t rhs_panel;  /* right-hand sides per CTA in the subdomain solve; 0 = measured: the
                           first DDM application of each batch size times every panel width
                           the context's solve kernel takes on the widest dependency level
                           and keeps the fastest (the twisted kernels: 8, fixed) */
    int32_t restart;    /* GMRES restart length; 0 = 30 */
    int32_t verbose;    /* 1: per-iteration residuals on stderr */
    void *stream;       /* cudaStream_t to run on; NULL = the library's own stream */
    int32_t profile;    /* 1: time every kernel launch with CUDA events (helm_profile_get) */
    int32_t tc_kernel;  /* HELM_PREC_TF32 and HELM_PREC_F16: 0 = tcgen05/TMEM kernels: the
                           two-ended ("twisted") kernel when every subdomain has at least 4
                           lines and blocks have at most 256 rows (384 with HELM_PREC_F16),
                           else the one-ended one for blocks of at most 256 rows, else
                           mma.sync; 1 = always mma.sync; 2 = tcgen05, one-ended form only */
    int32_t wait_limit; /* bound of every ordinary spin-wait inside the subdomain-solve
                           kernels (a bulk copy, an MMA commit, a peer CTA's handshake),
                           in polls of the mbarrier: 0 = default (2^22 polls); n > 0 = n
                           polls; -1 = no poll, so the first such wait gives up at once.  A wait that gives up makes the call return
                           HELM_ERR_TIMEOUT; the kernel stops issuing work, still waits
                           (with the default bound) for the copies and MMAs it has started,
                           frees its tensor memory and exits, so the CUDA context stays
                           usable.  -1 exists for testing callers' handling of that error. */
    int32_t sweep_order; /* 3D only (Section 4.1): 0 = the order (Sorder3D) of Algorithm
                           4.1, the 2D order with first +z then -z; 1 = the alternative
                           order given there, along which the L1 distance to the first
                           direction never decreases: (+,+,+), (-,+,+), (+,-,+), (+,+,-),
                           (-,-,+), (-,+,-), (+,-,-), (-,-,-).  The routing rules (4.1,
                           4.2, smallest usable later sweep) are the same.  Other values
                           return HELM_ERR_ARG. */
    int64_t max_device_bytes; /* cap on the device memory the context may hold (its own
                           allocations: coefficients, stencil, factors, work and staging
                           buffers); 0 = no cap.  An allocation that would go beyond it is
                           refused with HELM_ERR_OOM before cudaMalloc is called, and
                           helm_setup refuses a problem whose grid arrays alone exceed it
                           before touching the device. */
    int32_t algorithm;  /* 0 = the diagonal sweeps (Algorithm 3.1 in 2D, 4.1 in 3D, with
                           sweep_order); 1 = the additive DDM of Section 2.2 (Algorithm 2.1 in
                           2D, 2.2 in 3D): at every step s = 0 .. sum_k (nb_k - 1) every
                           subdomain solves with the transfers that left its neighbours at
                           step s - |d|_1 (all 3^n - 1 directions d), and the solution sums the
                           box-weighted local solutions of every step.  Same kernels; about
                           (sum_k (nb_k - 1) + 1) / 2^n times the solves of the sweeps.  Other
                           values return HELM_ERR_ARG. */
} helm_config;

typedef struct {
    int32_t iters;         /* GMRES iterations (max over right-hand sides) */
    int32_t applications;  /* DDM applications performed */
    double resid;          /* final relative residual |Jf - Au|/|Jf| (max over RHS) */
    double t_factor_ms;    /* last helm_factor wall time */
    double t_solve_ms;     /* this call's wall time */
    int32_t levels;        /* dependency levels of one DDM application */
    int32_t solves;        /* subdomain solves of one DDM application */
} helm_stats;

/* Create a context: copy m (squared slowness 1/c^2, float64, full grid,
 * host pointer; a NaN or infinite entry returns HELM_ERR_NUMERIC before any
 * device work), build the PML coefficients (Eq. 2.1-2.3), the subdomain
 * windows (Section 2.1), the routing table of transferred sources by Rules
 * 3.1/3.2 (2D) or 4.1/4.2 (3D) with the smallest-usable-sweep rule of
 * Algorithm 3.1/4.1, and the dependency levels of one sweep application.
 * ndim is 2 or 3; n[2] is ignored in 2D.  cfg may be NULL.  On success *out
 * owns all device memory of the problem. */
int helm_setup(helm_ctx **out, int ndim, const int64_t n[3], double h, double omega,
               const double *m, const helm_pml *pml, const helm_partition *part,
               const helm_config *cfg);

/* Factor every subdomain PML operator L_{ij} (the local problems of
 * Algorithm 3.1/4.1) as a block-tridiagonal block LU over lines (2D) or
 * planes (3D): S_1 = A_11, S_j = A_jj - diag(a_j) S_{j-1}^{-1} diag(c_{j-1}),
 * storing D_j = S_j^{-1} (dense, partial pivoting).  Idempotent. */
int helm_factor(helm_ctx *ctx);

/* One application of Algorithm 3.1 (2D) / 4.1 (3D) to sources F: returns
 * u_DDM = sum_l sum_ij beta_{0,0;ij} u^l_ij (Eq. 3.x/4.x).  In constant medium
 * this is the global PML solution up to subdomain-PML truncation (Theorems
 * 3.1/4.1).  F, U: complex128 [nrhs][full grid]. */
int helm_apply_ddm(helm_ctx *ctx, int nrhs, const void *F, void *U, int mem);

/* Solve the global PML system A u = J f for nrhs sources with FP64 flexible
 * GMRES, right-preconditioned by one DDM application per iteration
 * (Remark 1), restarted every cfg.restart iterations, until the relative
 * residual is <= rtol for every right-hand side or maxit iterations.
 * Returns HELM_ERR_NO_CONVERGENCE (with U and *st written) if maxit is hit.
 * When the whole batch does not fit in the free device memory (or under
 * cfg.max_device_bytes) with its window buffers and 2 restart + 2 Krylov
 * vectors per right-hand side, the call lowers the restart length (to no less
 * than 8) and then, if needed, solves the right-hand sides in consecutive
 * chunks; st then gives the largest iteration count and residual over the
 * chunks and their total of DDM applications.  st may be NULL. */
int helm_solve(helm_ctx *ctx, int nrhs, const void *F, void *U, int mem, double rtol,
               int maxit, helm_stats *st);

/* The DDM as a stationary iteration, the way Section 5.2.2 runs it (as an
 * iterative solver rather than a preconditioner, to show the residual decay
 * of the method itself): u_0 = 0, u_{k+1} = u_k + M (J f - A u_k) with M one
 * application of Algorithm 3.1/4.1, until the relative residual
 * |Jf - A u|/|Jf| is <= rtol for every right-hand side or maxit applications.
 * st->iters and st->applications give the applications made, st->resid the
 * last residual (max over right-hand sides).  Returns HELM_ERR_NO_CONVERGENCE
 * (with U and *st written) if maxit is hit.  F, U: complex128
 * [nrhs][full grid].  st may be NULL. */
int helm_iterate(helm_ctx *ctx, int nrhs, const void *F, void *U, int mem, double rtol,
                 int maxit, helm_stats *st);

/* Adjoint solve A^H lambda = g.  A is complex symmetric, so this runs
 * helm_solve on conj(g) with the same factors and DDM and conjugates the
 * result.  G, Lambda: complex128 [nrhs][full grid]. */
int helm_adjoint(helm_ctx *ctx, int nrhs, const void *G, void *Lambda, int mem, double rtol,
                 int maxit, helm_stats *st);

/* Gradient of L(m) = 1/2 sum_s |P u_s - d_s|^2 with respect to m:
 * grad_k = -omega^2 sum_s Re(conj(lambda_{s,k}) J_k u_{s,k}), from forward
 * fields U and adjoint fields Lambda (complex128 [nsrc][full grid]).  grad:
 * float64 full grid, overwritten. */
int helm_gradient(helm_ctx *ctx, int nsrc, const void *U, const void *Lambda, double *grad,
                  int mem);

/* FP64 residual R = J F - A U on the full grid (complex128 [nrhs][grid]). */
int helm_residual(helm_ctx *ctx, int nrhs, const void *F, const void *U, void *R, int mem);

/* Solve one subdomain PML problem L_s u = r (the local solve of Algorithm
 * 3.1/4.1) with its stored factors.  s indexes subdomains with x fastest;
 * R, U: complex128 [nrhs][window], the window being the subdomain's box plus
 * overlap plus PML (helm_window_info).  For testing the factor and solve. */
int helm_subdomain_solve(helm_ctx *ctx, int s, int nrhs, const void *R, void *U, int mem);

/* The same subdomain solve as helm_subdomain_solve, for callers that cannot
 * allocate device memory when they call it (code running inside an
 * allocator callback, a loop with a fixed device-memory budget, or a host
 * that has reserved all device memory up front).  The paper has no
 * counterpart; this is a property of the library, not of the method.
 * R and U are DEVICE pointers (complex128 [nrhs][window]) that the caller
 * owns; nothing is allocated or freed.  The solve runs on the kernel that
 * helm_subdomain_solve uses for the context's precision (the SIMT solve for
 * HELM_PREC_F64 and HELM_PREC_MIXED, the tensor-core solves for
 * HELM_PREC_TF32 and HELM_PREC_F16), so both entry points give the same
 * answer.  The working buffer lives in one static device array of 64 MiB that
 * every GPU loading the library holds until exit: nrhs times the window size
 * times 8 bytes (complex64 context) or 16 bytes (complex128 context) must fit
 * in 64 MiB - 256 bytes, else HELM_ERR_ARG with the sizes in
 * helm_last_error().  The current device must be the one that was current at
 * helm_setup, else HELM_ERR_ARG.  The first call on a device looks up that
 * array's device address (set-up work): make it before any stream capture;
 * after cudaDeviceReset the looked-up address is stale, so do not call this
 * again in that process.  Calls share the array and leave its contents
 * behind; calls whose GPU work overlaps race on it.  Synchronises the
 * context's stream before returning. */
int helm_subdomain_solve_noalloc(helm_ctx *ctx, int s, int nrhs, const void *R, void *U);

/* Window of subdomain s: lo[3], hi[3] full-grid node ranges (hi exclusive). */
int helm_window_info(helm_ctx *ctx, int s, int64_t lo[3], int64_t hi[3]);

/* Number of subdomains, full-grid size N[3] (N[2] = 1 in 2D). */
int helm_problem_info(helm_ctx *ctx, int64_t *nsub, int64_t N[3]);

/* Kernel classes reported by helm_profile_get. */
enum helm_kernel_class {
    HELM_K_FACTOR = 0,   /* block-Thomas factorisation */
    HELM_K_SOLVE = 1,    /* subdomain forward/backward solves */
    HELM_K_GATHER = 2,   /* local sources + transferred sources (Psi) */
    HELM_K_ASSEMBLE = 3, /* u_DDM = sum beta_00 u */
    HELM_K_KRYLOV = 4,   /* FP64 residual, J scaling and GMRES BLAS-1 */
    HELM_K_NCLASS = 5
};

/* Accumulated per-class counters since the last helm_profile_reset:
 * launches counts every kernel launch; ms is device time from CUDA events
 * recorded on the context's stream around each launch (only when
 * helm_config.profile = 1, else 0); bytes and flops are the algorithmic
 * DRAM bytes and floating-point operations of those launches (factor and
 * solve classes: dense block reads/writes and complex multiply-adds; the
 * solves count each block inverse at the factors' complex storage size, 8
 * bytes per entry for complex64 and 16 for complex128, also where the
 * tensor-core kernel streams a 4-byte FP16 image of it). */
typedef struct {
    int64_t launches[8];
    double ms[8];
    double bytes[8];
    double flops[8];
} helm_profile;

int helm_profile_reset(helm_ctx *ctx);
int helm_profile_get(helm_ctx *ctx, helm_profile *out);

/* Bytes of device memory held by the context. */
int64_t helm_device_bytes(helm_ctx *ctx);

/* Frees the context's subdomain factors (and their tile images) and its work
 * buffers (window buffers, Krylov vectors, staging), keeping everything
 * helm_setup built; the context is then unfactored.  helm_factor recomputes
 * the same factors (the factorization is deterministic), so a later solve or
 * adjoint gives bitwise the result it would have given before the release.
 * For a caller that must hold the device memory free between a forward solve
 * and its adjoint (Remark 2: the adjoint reuses the forward operator A(m),
 * so recomputing its factors is the alternative to keeping them).  Waits for
 * the context's stream.  Returns HELM_OK or HELM_ERR_ARG (null context). */
int helm_release(helm_ctx *ctx);

void helm_destroy(helm_ctx *ctx);
const char *helm_strerror(int code);
const char *helm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HELM_H */
