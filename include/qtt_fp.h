/*
 * qtt_fp.h -- C ABI of the GB300 QTT Fokker-Planck solver.
 *
 * The library time-steps the joint PDF f(phi1, phi2; x1, x2, x3) of the
 * reactive-scalar Fokker-Planck equation (paper: Eq. FP0, discretised as
 * Eq. FP2 with the zero-sum composition-space ghost rules of Eq. compBCs)
 * on a 2^K1 x ... x 2^K5 grid.  f is stored as a quantics tensor train
 * (matrix product state, paper: "Matrix product state encoding"): N = sum K_d
 * sites of physical dimension 2, dimension order phi1, phi2, x1, x2, x3, bits
 * of each dimension most significant first.  Finite-difference operators are
 * matrix product operators (paper: "Matrix product state algorithm").
 *
 * Conventions for every entry point:
 *   - Calls never abort or trap.  Each returns a qtt_status; on failure the
 *     context's last-error string (qtt_last_error) says why.
 *   - Host arrays passed in are owned by the caller and only read during the
 *     call (parameters are copied at init).  Output arrays are host FP64
 *     memory owned by the caller, written after the library's stream has
 *     been synchronised.
 *   - The library owns all device memory of a context.  A context is not
 *     thread-safe; use one context per host thread / stream.
 *   - All device work of a context runs on params.stream (NULL = the legacy
 *     default stream of the current device).
 */
#ifndef QTT_FP_H
#define QTT_FP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qtt_ctx qtt_ctx; /* opaque */

typedef enum {
  QTT_OK = 0,
  QTT_EINVAL = 1,   /* invalid argument or parameter */
  QTT_ENOMEM = 2,   /* device or host allocation failed */
  QTT_ECUDA = 3,    /* a CUDA runtime call failed */
  QTT_ENOCONV = 4,  /* an eigen / QR iteration hit its sweep cap */
  QTT_ETIMEOUT = 5, /* a bounded device wait gave up */
  QTT_ENAN = 6,     /* a non-finite value appeared in the state */
  QTT_ESTATE = 7,   /* call not valid in the context's current state */
  QTT_EIO = 8       /* checkpoint file error */
} qtt_status;

/* Arithmetic of the core contractions (MPO x MPS, Hadamard, sketches).
 * FP64: everything in FP64.  The reduced forms keep FP64 for the Gram
 * matrices and eigensolves of the SVD truncation and for all norm / mass
 * accumulation; their QR factorisations run in FP32 followed by one FP64
 * re-orthonormalisation step.  FP32: exact-slice bf16 tensor-core products
 * (3 x 3 slices, unbiased, ~2^-24 of the row maxima); TF32 and BF16X3 (hi/lo
 * split): tensor cores with FP32 accumulation.  Contractions with an
 * operator bond <= 32 run on the CUDA cores (FP32 in those three forms).
 * BF16X10: the products carrying the state as 4 x 4 exact bf16 slices cut
 * from the FP64 mantissa (10 slice products, exact FP32 accumulation,
 * ~2^-31 of the row maxima), except those of the mixing term (O(dt): its
 * product errors reach the state scaled by dt Omega), which take the 3 x 3
 * slices of FP32; the sketch products hi/lo TF32, the operator-bond
 * contractions that carry the state in FP64, those of the sketch in FP32. */
typedef enum { QTT_FP64 = 0, QTT_FP32 = 1, QTT_TF32 = 2, QTT_BF16X3 = 3, QTT_BF16X10 = 4 } qtt_precision;

typedef struct {
  int32_t bits[5];       /* K per dimension, order phi1, phi2, x1, x2, x3; 1..12 */
  int32_t chi_max;       /* maximum bond dimension chi (paper: Eq. MPSdofs) */
  double svd_rel_tol;    /* also drop singular values below tol * sigma_1 (0 = cap only) */
  int32_t precision;     /* qtt_precision */
  int32_t oversample;    /* extra sketch columns of the randomized rounding (<= 0: default 8) */
  int32_t exact;         /* 1: no truncation at all (requires chi_max >= 2^(N/2) and tol = 0) */
  uint64_t seed;         /* seed of the Gaussian sketches of the randomized rounding */
  double omega;          /* Omega_mix (constant) */
  double da;             /* Damkohler number: S_1 = S_2 = -da * phi1 * phi2 */
  double gamma;          /* diffusivity in x */
  double d_phi;          /* artificial composition-space dissipation (Eq. FP2) */
  double dt;             /* time step */
  double shear_amp;      /* u1 += shear_amp * tanh(x2 - pi) */
  int32_t n_umodes;      /* velocity Fourier modes: u_c += a sin(k . x + theta), k_c = 0 */
  const int32_t* umode_comp;   /* [n_umodes] component c in 0..2 */
  const int32_t* umode_k;      /* [3 * n_umodes] integer wavevectors */
  const double* umode_phase;   /* [n_umodes] */
  const double* umode_amp;     /* [n_umodes] */
  double ic_sigma;       /* std of the two composition-space Gaussians */
  double ic_blend_width; /* ic_kind 0: w(x2) = (1 + tanh((x2 - pi) / width)) / 2;
                            ic_kind 1: w(x1) = (tanh((x1 - pi/2) / width) - tanh((x1 - 3pi/2) / width)) / 2 */
  double ic_c_hi[2];     /* Gaussian centre used where w -> 1 */
  double ic_c_lo[2];     /* Gaussian centre used where w -> 0 */
  int32_t n_icmodes;     /* optional modulation f0 *= 1 + sum b cos(q . x + psi) */
  const int32_t* icmode_k;     /* [3 * n_icmodes] */
  const double* icmode_phase;  /* [n_icmodes] */
  const double* icmode_amp;    /* [n_icmodes] */
  int32_t rk_variant;    /* 0 = Heun (default), 1 = midpoint */
  int32_t flow;          /* 0: shear + seeded modes; 1: the paper's jet through a Taylor-Green
                            vortex (Eq. velField) on [0, l0)^3, l0 = 2 pi, k = 4 pi / l0, scale u0
                            (shear_amp unused; seeded modes, if any, are added) */
  double u0;             /* velocity scale of flow 1 */
  int32_t ic_kind;       /* 0: blend in x2 (above); 1: the paper's Gaussian step function in x1
                            (Eq. initPDF) smoothed by tanh edges of width ic_blend_width;
                            2 (no counterpart in the paper): a Gaussian of std ic_sigma whose
                            centre moves with x, c1 = ic_c_hi[0] + A sin(x1) cos(x2),
                            c2 = ic_c_hi[1] - A sin(x2 + x3), A = ic_blend_width >= 0, each factor
                            normalised on the phi grid; it couples phi with x, and is encoded
                            by tensor cross from point samples (paper: initial states by the
                            tensor-cross algorithm, "Computational complexity") */
  int32_t sgs;           /* 1: the subgrid closures of Eq. FP0 replace gamma and omega by fields:
                            gamma(x) = gamma + gamma_SGS(x), gamma_SGS = c_s Delta^2 / 2 *
                            sqrt(sum_ij (d_j u_i + d_i u_j)^2) (Smagorinsky; CFD2 derivatives of
                            the sampled velocity), the diffusion taken in flux form with face
                            values averaged from the two neighbours, and the mixing rate
                            Omega_mix(x) = c_omega gamma(x) / Delta^2 (LMSE); Delta = delta_cells
                            (h1 h2 h3)^(1/3); omega unused.  Needs K3 + K4 + K5 <= 18; not
                            available for qtt_grad */
  double c_s;            /* Smagorinsky constant (paper: 0.11) */
  double c_omega;        /* SGS mixing-rate constant C_Omega (paper: 0.25 .. 1) */
  double delta_cells;    /* filter width in cells (paper: 3) */
  int32_t moment_ref;    /* 1: also step the first-moment equation Eq. FPMoms with S = 0 (the
                            "numerically exact" <Phi_a>(x) of the error measures, Eqs. RMSE0/1)
                            on the dense x grid, by the same RK2 and CFD2 stencils (flux form
                            under sgs), from the initial <Phi_a>(x); K3 + K4 + K5 <= 26 */
  void* stream;          /* cudaStream_t or NULL (the context then creates its own stream) */
} qtt_params;

/* What qtt_observe returns (all FP64, space averages normalised by the
 * number of x points; paper Eqs. 2, spaceAvg, RACov, SGSCov). */
typedef enum {
  QTT_OBS_SCALARS = 0,   /* 13 values: time, norm_avg, mean1_avg, mean2_avg,
                            phi11_avg, phi22_avg, phi12_avg, R12, Y12,
                            product_J, discarded_weight (sum over the bonds of the
                            discarded squared singular values in the last step),
                            steps, norm2 (sum of f^2 over every grid cell) */
  QTT_OBS_BONDS = 1,     /* N+1 values: bond dimensions b_0..b_N (b_0 = b_N = 1) */
  QTT_OBS_DENSE = 2,     /* 2^N values: f[i1][i2][j1][j2][j3] row-major; N <= 26 */
  QTT_OBS_MEANS = 3,     /* 3 * 2^(K3+K4+K5) values: <1>(x), <Phi_1>(x), <Phi_2>(x); x row-major */
  QTT_OBS_POINTS = 4,    /* f at given multi-indices: pass in `out` n groups of N bits
                            (as doubles 0/1, MSB first per dimension), cap = n * N;
                            the first n entries are overwritten with the values */
  QTT_OBS_NVPP = 5,      /* 1 value: number of variables parameterising f (Eq. MPSdofs) */
  QTT_OBS_ERRORS = 7,    /* needs moment_ref = 1.  6 values, the space averages that the error
                            measures of Eqs. RMSE0 / RMSE1 take at one time sample:
                            avg <Phi_1> - 1/2, avg <Phi_2> - 1/2,
                            mean_x (<Phi_1>(x) - m_1(x))^2, mean_x (<Phi_2>(x) - m_2(x))^2
                            (m_a: the moment-equation reference), avg <Phi_1> - avg <Phi_2>,
                            mean_x (<1>(x) - 1)^2.  Over the time samples, E_t is the mean
                            of the squares of the first, second and fifth value and E_tx the
                            mean of the third, fourth and sixth; then Error_2b_up =
                            sqrt((E_t[1] + E_t[2]) / 2), Error_2b_down = sqrt((E_tx[3] +
                            E_tx[4]) / 2), Error_2c_up = sqrt(E_t[5]), Error_2c_down =
                            sqrt(E_tx[6]) */
  QTT_OBS_TIMINGS = 6    /* 20 values: for the kernel classes FP64 GEMM, QR, eigensolver,
                            other, tensor-core GEMM (incl. operand packing), CUDA-core GEMM
                            of the operator-bond contractions: launches, total ms,
                            algorithmic flops, recorded with CUDA events only when the
                            environment variable QTT_KERNEL_TIMING=1 was set at qtt_init
                            (zeros otherwise); then the number of kernels the library has
                            launched since it was loaded (always counted); then the
                            tensor-core flops as issued: algorithmic flops times the MMA
                            passes of each product's mode, TF32 passes counted twice (half
                            the bf16 rate), recorded like the classes */
} qtt_observable;

/* Build the initial PDF, velocity and operators (paper: "Flow case
 * definition"; encodings of "Matrix product state algorithm") and upload
 * them.  *out receives a new context (NULL on failure). */
qtt_status qtt_init(const qtt_params* params, qtt_ctx** out);

/* Advance nsteps explicit RK2 steps of Eq. FP2 in MPS form.  Each stage
 * forms f + dt L(f) as a sum of MPO x MPS products (linear operator) and a
 * Hadamard product with the conditional means (mixing drift), compresses it
 * by randomized rounding and truncates it by an SVD sweep to chi_max. */
qtt_status qtt_step(qtt_ctx* ctx, int32_t nsteps);

/* Discrete adjoint (paper: the observables of Eqs. 2 and spaceAvg; the
 * gradient is of the discretised Heun map of Eq. FP2, not of the continuous
 * equation).  Restarts the context from its initial PDF, takes nsteps Heun
 * steps and returns in out[0] the mean product J = avg_x (<1> - <Phi_1> -
 * <Phi_2>) of the final state and in out[1 ..] dJ/dtheta for theta = Omega,
 * Da, gamma, the amplitude of each velocity mode (params.umode_amp order)
 * and of each initial-condition mode (params.icmode_amp order), dt held
 * fixed: 1 + 3 + n_umodes + n_icmodes values (cap >= that, else QTT_EINVAL;
 * *written receives the count).  The backward sweep applies the transposed
 * stage operators (MPO transposes, the transposed mixing drift and the
 * transpose of its dependence through <Phi_a>) to the adjoint state and
 * rounds each adjoint stage to chi like a forward stage; in exact mode
 * nothing is rounded and the result is the exact gradient of the discrete
 * map.  Forward states are kept every ckpt_every steps (<= 0: only the
 * first) and each segment is recomputed before its backward sweep.  The
 * context is left at the final state (time nsteps * dt).  Heun only
 * (rk_variant 0). */
qtt_status qtt_grad(qtt_ctx* ctx, int32_t nsteps, int32_t ckpt_every, double* out, int64_t cap, int64_t* written);

/* Backward of the bond truncation (the derivative of the SVD rounding of
 * section "Matrix product state algorithm"), context-free, on the device.
 * The truncation is the simultaneous one of every bond that the stages use:
 * T(X) = Pi_1 ... Pi_{N-1} X, Pi_n the orthogonal projector onto the k_n
 * leading left singular vectors of X's unfolding at cut n (first n sites
 * against the rest), k_n = min(chi, #{lambda_i > max(tol^2, 1e-24)
 * lambda_0}) over the eigenvalues lambda of the cut's right Gram.  The call
 * returns (dT/dX)^T ybar, exact where every kept eigenvalue is separated
 * from the discarded ones; eps > 0 replaces each 1 / (lambda_i - lambda_j)
 * by its Lorentzian broadening (lambda_i - lambda_j) / ((lambda_i -
 * lambda_j)^2 + eps^2) (eps in the units of lambda, i.e. of |X|^2).  A kept
 * eigenvalue near the Gram's FP64 rounding (lambda_k below ~1e-12 lambda_0)
 * makes the exact weight 1 / lambda_k of the null-space part amplify that
 * rounding: pass tol >= 1e-7 or eps >= 1e-8 lambda_0 for such spectra.
 *   N       number of binary sites, 2 .. 64
 *   rx      host array of N + 1 bonds of x (rx[0] = rx[N] = 1, rx[n] <= 1024,
 *           rx[n] <= 2 rx[n-1])
 *   x       device array: the N cores of X, core n being [rx[n]][2][rx[n+1]]
 *           row-major (site 1, the most significant index, first), stored
 *           one after another; cores 0 .. N-2 left-orthonormal (each
 *           (2 rx[n]) x rx[n+1] matrix has orthonormal columns), which is not
 *           checked: otherwise the result is not the derivative
 *   sy, ybar  the cotangent as a train of any bonds sy (<= 1024), same layout
 *   xbar    device array receiving the result as a train of bonds 1,
 *           2 rx[1], ..., 2 rx[N-1], 1 in the same layout: site 1 [Q_1 D_1],
 *           site n [[Q_n D_n], [0 Q_n]], site N [[E], [x's last core]]; cap
 *           is its room in doubles, *written the count used
 *   kept    host array receiving the N - 1 kept counts k_n
 *   stream  CUDA stream (NULL: the legacy default stream); the call
 *           allocates and frees its work space and synchronises the stream
 * Returns QTT_EINVAL for bad sizes or pointers (no device work done; the
 * message names the check), QTT_ECUDA on a CUDA failure, QTT_ESTATE when the
 * eigen-decomposition reports a failure.  The paper rounds with an SVD but
 * does not differentiate it; this is the backward a discrete adjoint through
 * the truncated steps would use. */
qtt_status qtt_truncate_vjp(int32_t N, const int32_t* rx, const double* x, const int32_t* sy, const double* ybar,
                            int32_t chi, double tol, double eps, double* xbar, int64_t cap, int64_t* written,
                            int32_t* kept, void* stream);

/* Batched stepping of independent PDFs (no counterpart in the paper, which
 * steps one PDF): advances each of ctxs[0..n) by nsteps steps, enqueueing the
 * work of every context before synchronising any of them, so that contexts
 * on different streams (a context created with stream NULL owns one) run
 * concurrently on the GPU.  Once every context has captured its step graphs
 * (after its first three steps), each step is one launch of a graph that
 * embeds every context's step graph as an independent node; it is built the
 * first time a set of contexts is stepped together and rebuilt when the set,
 * a context's graphs or the contexts' relative step parity change (the
 * contexts must belong to the current device).  The
 * contexts may differ in grid, chi, coefficients and precision; a context
 * must not appear twice.  Returns QTT_OK, or the status of the first context
 * (lowest index) that failed, whose index goes to *failed (-1 when none;
 * failed may be NULL); the other contexts have still been advanced.
 * Results are identical to stepping each context alone. */
qtt_status qtt_step_many(qtt_ctx* const* ctxs, int32_t n, int32_t nsteps, int32_t* failed);

/* Extract observables (see qtt_observable).  `out` has room for `cap`
 * doubles; *written receives the number written.  Returns QTT_EINVAL when
 * cap is too small. */
qtt_status qtt_observe(qtt_ctx* ctx, int32_t what, double* out, int64_t cap, int64_t* written);

/* Relative L2 distance ||a - b|| / ||b|| of the two states (same grid),
 * from FP64 overlaps <a|a>, <b|b>, <a|b>. */
qtt_status qtt_compare(qtt_ctx* a, qtt_ctx* b, double* rel_l2);

/* Checkpoint: cores, bonds, time and step count, with a header and an
 * FNV-1a checksum.  Load requires a context initialised with the same grid. */
qtt_status qtt_save(qtt_ctx* ctx, const char* path);
qtt_status qtt_load(qtt_ctx* ctx, const char* path);

/* Allocation-free variant of qtt_observe(ctx, QTT_OBS_POINTS, ...), same
 * arguments and result: inout holds n groups of N index bits (doubles 0/1,
 * most significant bit first per dimension), cap = n * N, and the first n
 * entries receive f at those points.  The paper has no counterpart.  It
 * serves callers that cannot allocate device memory during the call: a
 * process whose device memory is entirely held by its own pool allocator, or
 * a per-step monitoring loop that cannot pay cudaFree's implicit device-wide
 * synchronisation.  The call copies the query in and the values out on the
 * context's stream and synchronises that stream before returning.  The query,
 * scratch and results use one 4 MiB device array fixed at compile time and
 * shared by the whole process, which limits a call to
 * floor((4 MiB - 768) / (8 + 8 N + 16 B)) points, B the largest bond the
 * context works with: chi_max + oversample for a truncating context (about
 * 1670 points at N = 40, chi_max 128), 2^floor(N/2) in exact mode (about 250
 * at N = 20).  Larger requests return QTT_EINVAL, the message giving the
 * limit.  The first call on a device looks up that array's device address
 * (with the device current); make that first call before any stream capture.
 * Calls whose work overlaps on the GPU race on the shared array: serialise
 * them. */
qtt_status qtt_observe_points_noalloc(qtt_ctx* ctx, double* inout, int64_t cap, int64_t* written);

void qtt_destroy(qtt_ctx* ctx);

/* Last error message of ctx; with ctx NULL, that of the calling thread's last
 * failed call that takes no context (qtt_init, qtt_truncate_vjp,
 * qtt_host_dense, qtt_selftest). */
const char* qtt_last_error(const qtt_ctx* ctx);

/* Library version string. */
const char* qtt_version(void);

/* ---------------------------------------------------------------------
 * Host-side verification entry points.  They run the initialisation's
 * encoders on the CPU only (no GPU, no context) so that the operator and
 * state encodings can be checked against independent dense constructions.
 *
 * qtt_host_dense writes a dense expansion of one object built from params:
 *   0        initial PDF f0 (paper: "Flow case definition" with the workload's
 *            initial condition), 2^N values, N <= 26
 *   1, 2, 3  velocity component u_1, u_2, u_3 over x, 2^(K3+K4+K5) values
 *   10 + d   first-derivative operator of dimension d (0..4) as a row-major
 *            M_d x M_d matrix: zero-sum ghosts of Eq. compBCs for d < 2,
 *            periodic CFD2 for d >= 2
 *   20 + d   second-derivative operator of dimension d, same conventions
 *   30       W_lin, the linear part of the right-hand side of Eq. FP2
 *            (2^N x 2^N, N <= 12)
 *   31       the stage operator I + dt W_lin (2^N x 2^N, N <= 12)
 *   32       the composition-space factor of the mixing term,
 *            -dt Omega D1phi_a, for a = 1, 2: 2 x (M1 M2)^2 values (with sgs:
 *            -dt D1phi_a, the rate then being the x factor of item 33)
 *   33       sgs only: the encoded mixing rate Omega_mix(x), 2^(K3+K4+K5) values
 *   40       bond dimensions of the stage operator (N + 1 values)
 *   41       bond dimensions of the encoded initial PDF (N + 1 values)
 *   42       sgs only: bond dimensions of the Omega_mix(x) train (K3+K4+K5+1 values)
 * Returns QTT_EINVAL for an unknown `which`, invalid params or cap too small.
 * ------------------------------------------------------------------- */
qtt_status qtt_host_dense(const qtt_params* params, int32_t which, double* out, int64_t cap, int64_t* written);

/* Device self-checks of the kernel families on seeded random operands
 * (needs a GPU; no context).  The paper has no counterpart: these check the
 * implementation, not the method.  Values written (then one error-flag word):
 *   0  tensor-core GEMM: for 7 shapes x 6 modes (BF16X3, TF32, TF32X3, BF16, BF16X6, BF16X10)
 *      max |C_tc - C_fp64| / max |C_fp64| (-1 when a shape is not supported)
 *   1  Householder QR: for 13 shapes x (FP64, FP32, FP32 followed by one
 *      FP64 Newton-Schulz step) the orthogonality max |Q^T Q - I| and the
 *      projection residual ||Y - Q Q^T Y|| / ||Y||
 *   2  eigensolver: for 11 (size, spectrum) cases x (FP64, FP32)
 *      max |G U - U diag(lam)| / max |G|, max |U^T U - I| and 1 if the
 *      eigenvalues are not descending; cases (136, 64, 7, 1, 200 with the
 *      graded spectrum 10^(-6 k / n)), then (136, rank 20), (136, a 40-fold
 *      eigenvalue), (136, graded to 1e-30), (200, rank 20), (200, graded to
 *      1e-30), (520, graded)
 *   3  accumulation bias of the tensor-core GEMM: positive operands, K = 32,
 *      256, 2048, modes (TF32X3, BF16X3), accumulation (one FP32 accumulator,
 *      FP64 sum of per-k-block accumulators): mean signed and max relative error
 *   4  throughput of the tensor-core GEMM on square products n = 4096, 8192
 *      in modes BF16 and BF16X3 (calls including the operand packing): per
 *      case n, the mode's enum value (BF16 3, BF16X3 0), TFLOP/s at 2 n^3 per
 *      call, and the max of |C - C_fp64| / sum_k |A_ik B_kj| over 16 sampled
 *      entries (needs ~3 GiB of device memory)
 *   5  tensor-core GEMM on seeded operands, for a check on the host: per case
 *      a header (M, N, K, outer, inner, A transposed, B transposed, beta;
 *      alpha = 1.5), A, B and the initial C as stored (batch-major; row-major,
 *      or column-major when transposed), then C after each of the modes
 *      BF16X3, TF32, TF32X3, BF16, BF16X6, BF16X10 (NaN where a mode does
 *      not take the shape); four cases, about 10.6 million values
 *   6  FP64 arithmetic throughput of the GPU: TFLOP/s of DFMA on the CUDA
 *      cores and of mma.sync m8n8k4 f64 (each the best of three launches of
 *      8 blocks of 256 threads per SM, 2 flops per FMA), the SM count and
 *      the number of blocks */
qtt_status qtt_selftest(int32_t which, double* out, int64_t cap, int64_t* written);

#ifdef __cplusplus
}
#endif

#endif /* QTT_FP_H */
