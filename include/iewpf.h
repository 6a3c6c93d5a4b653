/*
 * iewpf.h - C ABI of the GB300 implementation of the two-stage implicit
 * equal-weights particle filter (IEWPF) for a rotating shallow-water ocean
 * model with drifter and mooring observations (arXiv 1910.01031).
 *
 * All calls return IEWPF_OK (0) or a negative error code; a message for the
 * last error of a context is available from iewpf_last_error().  No C++
 * exception crosses this interface.  A NULL context gives IEWPF_EINVAL.
 *
 * Memory: a context owns every device buffer it allocates.  Host pointers
 * passed in are read (or written) during the call only.  Device pointers
 * passed in are borrowed for the duration of the call and are used on the
 * context's stream; the context never frees caller memory.
 *
 * Layouts: a field is [ny][nx] with x fastest; a particle state is
 * [3][ny][nx] holding (eta, hu, hv); an ensemble is [N_e][3][ny][nx] float32.
 * Positions are metres, unwrapped (a drifter that crosses the periodic
 * boundary keeps counting); the cell of (x, y) is
 * (floor(x/dx) mod nx, floor(y/dy) mod ny).
 *
 * Threading: a context is not thread-safe; different contexts may be used
 * from different threads.  All work of a context runs on its own CUDA stream.
 */
#ifndef IEWPF_H
#define IEWPF_H

#include <stdint.h>

#if defined(__GNUC__)
#define IEWPF_API __attribute__((visibility("default")))
#else
#define IEWPF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define IEWPF_OK 0
#define IEWPF_EINVAL (-1)      /* invalid argument or call order            */
#define IEWPF_ENOMEM (-2)      /* device or host allocation failed          */
#define IEWPF_ECUDA (-3)       /* a CUDA runtime call or launch failed      */
#define IEWPF_ENONFINITE (-4)  /* NaN/Inf met in the state or the weights   */
#define IEWPF_EBETA (-5)       /* beta < 0 (eq. betaTwoStage): N_y too large for N_psi */
#define IEWPF_EDOMAIN (-6)     /* Lambert W / alpha solve out of domain     */
#define IEWPF_ETIMEOUT (-7)    /* a bounded device wait gave up             */
#define IEWPF_ENOTPD (-8)      /* HQH^T + R not positive definite           */

#define IEWPF_OBS_DRIFTER 0
#define IEWPF_OBS_MOORING 1

/* Analysis schemes (App. A).  Two-stage: w_target = mean c_i, common beta,
 * nu perpendicular to xi (eqs. betaTwoStage, cistarTwoStage,
 * updateEquationTwoStageAgain).  One-stage: the original IEWPF,
 * w_target = max c_i and no nu (eqs. iewpf_targetWeight, iewpfCStar,
 * iewpfUpdateAgain). */
#define IEWPF_TWO_STAGE 0
#define IEWPF_ONE_STAGE 1

/* Problem description (Secs. 3.1-3.3 and 5 of the paper).
 * Grid: periodic nx x ny cells of dx x dy metres (eq. cell_center).
 * Physics: gravity g, Coriolis parameter f, constant equilibrium depth H_eq
 * (eq. swe_full).  theta: parameter of the generalized minmod limiter of the
 * reconstruction (1 <= theta <= 2).  courant: factor in front of the
 * 1/4 min(dx/a, dy/b) limit of eq. swecfl.  dt_model: the model step dt,
 * subdivided into as many scheme steps as the CFL condition requires.
 * Model error (Sec. 3.2): coarse grid of every c_omega-th cell (odd), SOAR
 * amplitude q0 (m) and length scale L0 (m), cut-off 2 coarse cells.
 * seed: key of the counter-based random numbers.
 * Observations: obs_kind, at most n_obs_max per cycle, standard deviation
 * obs_sigma in hu/hv units (m^2/s), R = obs_sigma^2 I.  dense_S = 1 keeps
 * the couplings between nearby observations in HQH^T (dense (HQH^T+R),
 * Cholesky in FP64); 0 keeps only each observation's 2x2 block as the paper
 * does (Sec. 4.2).  n_drifters_max: drifters each particle may carry in a
 * forecast (0 for none).  scheme: IEWPF_TWO_STAGE (0, the paper's method of
 * choice) or IEWPF_ONE_STAGE (App. A); other values give IEWPF_EINVAL. */
typedef struct {
    int nx, ny;
    double dx, dy;
    double g, f, H_eq;
    double theta;
    double courant;
    double dt_model;
    int c_omega;
    double q0, L0;
    uint64_t seed;
    int n_particles;
    int obs_kind;
    int n_obs_max;
    double obs_sigma;
    int dense_S;
    int instance_id;
    int n_drifters_max;
    int scheme;
} iewpf_params_t;

/* One observation time (Sec. 3.3).  xy: [n_obs][2] observed positions;
 * value: [n_obs][2] observed (hu, hv) in m^2/s, i.e. eq. drifterObservation
 * or eq. buoyObservation including the observation error.  For moorings the
 * positions must be the ones given to iewpf_create (xy may be NULL).
 * Drifters may instead give value = NULL with their previous fixes xy_prev
 * ([n_obs][2]) taken dt seconds earlier: the library then forms
 * eq. drifterObservation itself, as iewpf_drifter_obs does.  xy_prev and dt
 * are ignored when value is given. */
typedef struct {
    int n_obs;
    const double* xy;
    const double* value;
    const double* xy_prev;
    double dt;
} iewpf_obs_t;

/* Per-cycle diagnostics of iewpf_assimilate (App. A).  Each array has
 * N_e entries and may be NULL. */
typedef struct {
    double c_bar;        /* mean c_i (two-stage: also w_target)              */
    double beta;         /* eq. betaTwoStage; 0 for the one-stage scheme     */
    double* phi;         /* eq. iewpfPhi                                     */
    double* c;           /* eq. iewpf_ci, -log w^{n-1} = log N_e             */
    double* gamma;       /* eq. scalingGammaZeta                             */
    double* zeta;        /* eq. scalingGammaZeta                             */
    double* alpha;       /* eq. iewpfAlphaSol                                */
    double* neglogw;     /* final -log w_i, equal to w_target for every i    */
    double w_target;     /* mean c_i (two-stage) or max c_i (one-stage)      */
} iewpf_diag_t;

typedef struct iewpf_ctx iewpf_ctx_t;

/* Create a context: validates the parameters, allocates the ensemble (two
 * state buffers), precomputes the pull stencils of a unit hu/hv observation
 * (eq. detailedOPDUpdate), the 49x49 local block root (eq. Psquareroot,
 * Fig. localsvd) and, for moorings, factors HQH^T + R (eq. S_extended) in
 * FP64 on the GPU.  mooring_xy: [n_obs_max][2] for obs_kind = MOORING,
 * else NULL.  Errors: EINVAL (bad sizes: nx, ny must exceed 14 c_omega + 1;
 * c_omega odd; positive spacings, depth, step), ENOMEM, ECUDA, ENOTPD.
 * The state is zero until iewpf_set_state. */
IEWPF_API int iewpf_create(const iewpf_params_t* params, const double* mooring_xy, iewpf_ctx_t** out);

/* Free every resource of the context (a service of the library, not a step
 * of the method).  NULL is accepted and returns IEWPF_OK. */
IEWPF_API int iewpf_destroy(iewpf_ctx_t* ctx);

/* Copy the ensemble in ([N_e][3][ny][nx] float32; the state psi of Sec. 2,
 * fields (eta, hu, hv) of Sec. 3.1).  on_device: src is a device pointer
 * (copied on the context stream, after `stream` if given), else host
 * memory.  Clears the CFL rates kept from the last update.
 * Errors: EINVAL (NULL pointer), ECUDA. */
IEWPF_API int iewpf_set_state(iewpf_ctx_t* ctx, const float* src, int on_device, void* stream);

/* Copy the ensemble out ([N_e][3][ny][nx] float32), to device memory when
 * on_device (ordered after the context's work and before `stream`), else to
 * host memory.  Errors: EINVAL (NULL pointer), ECUDA. */
IEWPF_API int iewpf_get_state(iewpf_ctx_t* ctx, float* dst, int on_device, void* stream);

/* Ensemble forecast (eq. model_equation): n_model_steps model steps of
 * dt_model.  Each step picks n_sub = ceil(dt / dt_cfl) scheme steps per
 * particle from the CFL condition (eq. swecfl), runs them (advecting the
 * particle's drifters after each, if any are set), then adds the model
 * error Q^{1/2} xi (eq. model_error) when add_model_error != 0.  The model
 * error of step k uses draw counter = the context's model-step counter,
 * which advances by one per model step.  The call runs as one CUDA graph
 * (captured at the first call with its pattern of steps, model error and
 * drifters, then replayed): the scheme steps of a model step loop on the
 * device while the index is below the largest n_sub, so no host
 * synchronisation sits between model steps; the call returns after one at
 * the end.  Errors: EINVAL, ECUDA, ENONFINITE (checked once per call; also
 * when a CFL count exceeds 100 000 scheme steps, which caps the loop). */
IEWPF_API int iewpf_forecast(iewpf_ctx_t* ctx, int n_model_steps, int add_model_error);

/* As iewpf_forecast (eq. model_equation) but with a fixed number of scheme
 * steps per model step (n_sub > 0) for every particle, skipping the CFL
 * evaluation of eq. swecfl.  Errors: EINVAL (n_sub < 1, n_model_steps < 0),
 * ECUDA, ENONFINITE. */
IEWPF_API int iewpf_forecast_fixed(iewpf_ctx_t* ctx, int n_model_steps, int add_model_error, int n_sub);

/* One two-stage IEWPF analysis of the current ensemble against `obs`
 * (Sec. 4, steps 1-6; App. A): innovations and S d (FP64), c_i, the
 * perpendicular random vectors and gamma_i, zeta_i, the ensemble-wide
 * target weight and beta, alpha_i from the Lambert W function, and one
 * fused update psi <- psi + Q H^T S d + P^{1/2}(beta^{1/2} nu + alpha^{1/2}
 * xi) (eq. optUpdateEquationTwoStage); with params.scheme = IEWPF_ONE_STAGE
 * the one-stage analysis of App. A instead (w_target = max c_i, no nu).
 * Random draws use the context's cycle counter, which then advances by one.
 * diag may be NULL.
 * Errors: EINVAL (n_obs > n_obs_max, NULL values, a non-finite observed
 * value or position: refused before any device work, the state unchanged),
 * EBETA, EDOMAIN, ENONFINITE, ENOTPD, ECUDA. */
IEWPF_API int iewpf_assimilate(iewpf_ctx_t* ctx, const iewpf_obs_t* obs, iewpf_diag_t* diag);

/* Drifter observations from two GPS fixes (Sec. 3.3, eq. drifterObservation):
 * value[d] = ((x_d - x_prev_d) / dt * H_eq, (y_d - y_prev_d) / dt * H_eq),
 * each displacement taken by the minimum image on the periodic domain of
 * params (nx dx by ny dy metres), so a drifter that crossed the boundary
 * moves by its short way round.  Host arithmetic in FP64, no device work.
 * xy, xy_prev: host [n][2] metres; value: host [n][2] m^2/s.
 * Errors: EINVAL (NULL pointers, n < 0, dt not positive, non-finite input). */
IEWPF_API int iewpf_drifter_obs(const iewpf_params_t* params, int n, const double* xy, const double* xy_prev,
                                double dt, double* value);

/* Weights of the standard particle filter (Sec. 2.1, eqs.
 * standardParticleFilter and standardParticleFilterWeight) for the current
 * ensemble against subsets of one observation set, and how many particles
 * residual resampling would keep for sure (normalised weight above 1/N_e,
 * the count of the collapse experiment, Sec. 5.3).  The state is unchanged.
 *   obs      as for iewpf_assimilate; the innovations are those of
 *            eq. etaCompensatedInnovation.
 *   r_scale  R = r_scale * obs_sigma^2 I (the experiment uses 1 and 10).
 *   sets     host [n_sets][set_size] observation indices in [0, n_obs);
 *            1 <= set_size <= n_obs.  A subset may repeat an index.
 *   w        host [n_sets][N_e] normalised weights, or NULL.
 *   n_kept   host [n_sets]: particles with w_i > 1/N_e.
 * Per subset, w_i = exp(-(l_i - min l)) / sum_j exp(-(l_j - min l)) with
 * l_i = |d_i on the subset|^2 / (2 r_scale obs_sigma^2), in FP64.  Device
 * scratch of n_sets x (set_size x 4 + N_e x 8 + 4) bytes is allocated and
 * freed by the call.  Errors: EINVAL (bad subsets or observations),
 * ENOMEM, ECUDA. */
IEWPF_API int iewpf_sir_weights(iewpf_ctx_t* ctx, const iewpf_obs_t* obs, double r_scale, int n_sets,
                                int set_size, const int* sets, double* w, int* n_kept);

/* Ranks of observed values within the ensemble (Sec. 5.1, rank histograms):
 * for point m (cell cells[m] = (j, k), 0 <= j < nx, 0 <= k < ny) and
 * component c (0: hu, 1: hv), ranks[m][c] = #{i : (hu or hv)_i at the cell
 * + obs_sigma eps_{i,m,c} < y[m][c]}, in 0..N_e: the position the observed
 * value takes in the sorted list of the members perturbed by the
 * observation error.  eps_{i,m,c} is the FP64 normal number 2m + c of
 * particle i in Philox stream 3 (+ 16 x instance_id), draw `draw`.  All
 * arrays are host memory: cells [n_pts][2], y [n_pts][2], ranks [n_pts][2].
 * The state is unchanged.  Errors: EINVAL (a point outside the grid or a
 * non-finite value), ENOMEM, ECUDA. */
IEWPF_API int iewpf_rank(iewpf_ctx_t* ctx, int n_pts, const int* cells, const double* y, uint32_t draw,
                         int* ranks);

/* Drifters carried by every particle (Sec. 3.3, forward Euler with the
 * velocity hu/(H+eta) of the containing cell after each scheme step).
 * xy: [N_e][n][2] float64 unwrapped positions (host); n <= n_drifters_max.
 * n = 0 removes them.  get: the current positions into xy ([N_e][n][2]).
 * Errors: EINVAL (n out of range, NULL xy with n > 0), ECUDA. */
IEWPF_API int iewpf_set_drifters(iewpf_ctx_t* ctx, const double* xy, int n);
IEWPF_API int iewpf_get_drifters(iewpf_ctx_t* ctx, double* xy);

/* Drift trajectory forecast (Sec. 5.2): places drifters xy0 ([n][2]) in
 * every particle, runs `hours` of model steps with model error and stores
 * positions every out_every_s seconds (and at t = 0) into
 * traj[n_out][N_e][n][2], n_out = floor(hours*3600/out_every_s) + 1.
 * use_surrogate = 0 runs the plain stepper; 1 runs the surrogate attached
 * with iewpf_set_surrogate, k model steps per call (out_every_s must then be
 * a multiple of k dt_model), the plain stepper taking over for any k steps
 * whose surrogate state is not finite. */
IEWPF_API int drifter_forecast(iewpf_ctx_t* ctx, const double* xy0, int n, double hours,
                     double out_every_s, double* traj, int use_surrogate);

/* Drift forecast with its error measures (Sec. 5.2, eqs.
 * errorPerEnsembleDrifter and errorNorm), computed on the GPU: as
 * drifter_forecast, and at every output time t (t = 0 included)
 * E(t) = sqrt(mean_d mean_i |x_{i,d} - x_true,d|^2) against truth
 * ([n_out][n][2], unwrapped positions) and RMSE(t), the same with the
 * ensemble-mean position in place of the truth, into E[n_out] and
 * RMSE[n_out] (FP64).  traj ([n_out][N_e][n][2]) may be NULL; use_surrogate
 * as for drifter_forecast. */
IEWPF_API int drifter_forecast_errors(iewpf_ctx_t* ctx, const double* xy0, int n, double hours, double out_every_s,
                                      const double* truth, double* E, double* RMSE, double* traj, int use_surrogate);

/* Checkpoint (a service of the library): raw state, drifters and the two
 * draw counters written to / read from a host file; because the random
 * numbers are counter-based (Philox), a resumed run is bit-identical.  load
 * needs a context of the same sizes.  Errors: EINVAL (NULL path, file not
 * readable or writable, a checkpoint of other sizes or truncated), ECUDA. */
IEWPF_API int iewpf_save(const iewpf_ctx_t* ctx, const char* path);
IEWPF_API int iewpf_load(iewpf_ctx_t* ctx, const char* path);

/* Draw counters: model steps taken (the draw index of the model error,
 * eq. model_error) and cycles assimilated (the draw index of xi and nu,
 * App. A).  Either output pointer may be NULL.  Errors: EINVAL (NULL ctx). */
IEWPF_API int iewpf_get_counters(const iewpf_ctx_t* ctx, uint32_t* model_step, uint32_t* cycle);
IEWPF_API int iewpf_set_counters(iewpf_ctx_t* ctx, uint32_t model_step, uint32_t cycle);

/* Scheme steps each particle took in the last model step ([N_e] ints,
 * host), n_sub of eq. swecfl.  Errors: EINVAL (NULL), ECUDA. */
IEWPF_API int iewpf_last_nsub(const iewpf_ctx_t* ctx, int* n_sub);

/* Message of the last error of ctx ("" if none); static text for NULL. */
IEWPF_API const char* iewpf_last_error(const iewpf_ctx_t* ctx);

/* ---- building blocks, exposed for verification --------------------- */

/* Raw Philox4x32-10 blocks (Salmon et al., SC'11) computed on the GPU:
 * block b of counter (b, p, t, stream) with key (seed lo, seed hi).
 * out: host [n_blocks][4] uint32.  The model-error, xi and nu draws use
 * streams 0, 1, 2 and the rank perturbations stream 3 (plus 16 x
 * instance_id). */
IEWPF_API int iewpf_philox_blocks(uint64_t seed, uint32_t p, uint32_t t, uint32_t stream,
                        int64_t n_blocks, uint32_t* out);

/* Standard normals from those blocks by the Box-Muller pairing (the xi of
 * eq. model_error and App. A), computed on the GPU in FP64 (out64) and
 * FP32 (out32), host arrays of n; either may be NULL, not both.
 * Errors: EINVAL, ENOMEM, ECUDA. */
IEWPF_API int iewpf_normals(uint64_t seed, uint32_t p, uint32_t t, uint32_t stream, int64_t n,
                  double* out64, float* out32);

/* The ensemble-wide step of the two-stage IEWPF on the GPU (App. A,
 * eqs. betaTwoStage, cistarTwoStage, iewpfAlphaSol): from host arrays c,
 * gamma, zeta ([ne]) and N_psi, returns c_bar and beta in out2[2] and
 * alpha, c* and -log w in host arrays of ne (neglogw may be NULL).
 * Errors: EINVAL, EBETA, EDOMAIN, ENONFINITE, ENOMEM, ECUDA. */
IEWPF_API int iewpf_weights(int ne, double N_psi, const double* c, const double* gamma,
                  const double* zeta, double* out2, double* alpha, double* cstar,
                  double* neglogw);

/* The ensemble-wide step of the one-stage IEWPF on the GPU (App. A, eqs.
 * iewpf_targetWeight, iewpfCStar, iewpfAlphaSol): from host arrays c and
 * gamma ([ne]) and N_psi, returns w_target = max c_i and 0 (no beta) in
 * out2[2] and alpha, c* = w_target - c_i and -log w in host arrays of ne
 * (neglogw may be NULL).
 * Errors: EINVAL, EDOMAIN, ENONFINITE, ENOMEM, ECUDA. */
IEWPF_API int iewpf_weights_one_stage(int ne, double N_psi, const double* c, const double* gamma,
                                      double* out2, double* alpha, double* cstar, double* neglogw);

/* alpha of the one-stage IEWPF from the incomplete-gamma form of the
 * implicit equation (App. A, eq. numericalEqForAlpha), which keeps the
 * derivative term that the Lambert-W solution (eq. iewpfAlphaSol) drops:
 * P(N_psi/2, alpha_i gamma_i/2) = exp(-c*_i/2) P(N_psi/2, gamma_i/2), P the
 * regularised lower incomplete gamma function, solved on the GPU in FP64
 * with logarithms throughout (no overflow for large N_psi; the cost grows
 * like sqrt(N_psi)).  gamma ([ne], > 0) and cstar ([ne], >= 0) are host
 * arrays; alpha (host, [ne]) receives values in (0, 1], exactly 1 where
 * c* = 0.  Errors: EINVAL (bad arguments), EDOMAIN (no convergence or alpha
 * below the FP64 range), ENOMEM, ECUDA. */
IEWPF_API int iewpf_alpha_gamma(int ne, double N_psi, const double* gamma, const double* cstar,
                                double* alpha);

/* Largest ensemble iewpf_weights_noalloc accepts. */
#define IEWPF_WEIGHTS_NOALLOC_MAX_NE 4096

/* iewpf_weights for callers that cannot allocate device memory.  The paper
 * has no counterpart: this is a service of the library, not a step of the
 * method.  Some callers may not call cudaMalloc: hosts whose device memory
 * belongs to a pooling allocator (a framework's caching allocator that must
 * see every allocation), and latency-bound loops where cudaMalloc's implicit
 * device synchronisation is not acceptable.  This entry point computes the
 * same results as iewpf_weights (same kernel, same arguments and errors) but
 * allocates nothing: it calls no cudaMalloc, cudaFree or allocating library
 * routine.  Its scratch is a fixed array of 6 x 4096 + 8 doubles (about
 * 192 KiB) in the library's device memory, which every GPU that loads the
 * library holds until the process exits.
 *   - ne must not exceed IEWPF_WEIGHTS_NOALLOC_MAX_NE (4096); larger ensembles
 *     get IEWPF_EINVAL before any GPU work.
 *   - Every call looks up the scratch's device address with
 *     cudaGetSymbolAddress on the current device; no address is cached, so a
 *     context that was reset and created again is handled.
 *   - It must not be called while any stream capture is active on the
 *     device: its synchronous copies on the legacy default stream are not
 *     allowed during a capture.
 *   - Every call shares the one array, which keeps the last call's contents;
 *     the call clears its error flag itself.  Calls whose GPU work overlaps
 *     (from several host threads) race on the array: serialise them.
 *   - Inputs and outputs are host arrays, copied synchronously on the legacy
 *     default stream of the current device. */
IEWPF_API int iewpf_weights_noalloc(int ne, double N_psi, const double* c, const double* gamma,
                                    const double* zeta, double* out2, double* alpha, double* cstar,
                                    double* neglogw);

/* The context's precomputed pull stencils (eq. detailedOPDUpdate for a
 * unit observation): K[2][3][2R+1][2R+1] float64 (host), R = 7 c_omega
 * (unit hu, unit hv observation; fields eta, hu, hv).  Errors: EINVAL. */
IEWPF_API int iewpf_pull_stencil(const iewpf_ctx_t* ctx, double* K);

/* The context's 49x49 local block root U Sigma^{1/2} (eq. Psquareroot,
 * Sec. 4.6; row-major float64, host; block entries ordered
 * (dy+3)*7 + (dx+3)).  Errors: EINVAL. */
IEWPF_API int iewpf_local_block(const iewpf_ctx_t* ctx, double* M);

/* Levels of the local blocks of Sec. 4.6: block l is the 7 x 7 coarse
 * points around the centre block0[l] = (a, b) (host int[nobs][2], coarse
 * indices on the periodic nRx x nRy grid).  level[l] (host int[nobs]) = 0
 * when block l shares no coarse point with an earlier block, else one more
 * than the highest level among the earlier blocks it shares a point with.
 * Blocks of one level commute, so applying the levels in turn gives the
 * result of applying the blocks in observation order; the analysis of a
 * fixed (mooring) layout does so.  Host arithmetic only (no device).
 * Errors: EINVAL (nobs < 0, NULL arrays with nobs > 0, nRx or nRy < 1, a
 * centre outside the grid). */
IEWPF_API int iewpf_block_levels(const int* block0, int nobs, int nRx, int nRy, int* level);

/* Add Q^{1/2} x to every particle for coarse fields x ([N_e][N_R] float32,
 * host), the operator of eq. covarianceOperatorsDef (testing aid).
 * Errors: EINVAL (NULL x), ECUDA. */
IEWPF_API int iewpf_add_qhalf(iewpf_ctx_t* ctx, const float* x);

/* The CUDA stream (cudaStream_t) on which all work of ctx runs, so that a
 * caller can order its own work or record timing events on it (a service of
 * the library).  Errors: EINVAL. */
IEWPF_API int iewpf_stream(const iewpf_ctx_t* ctx, void** stream);

/* n scheme steps (eq. swecfl's subdivision of the model step) of length dt
 * seconds for every particle, without the CFL evaluation, the model error
 * or any host synchronisation: the bare stepper (Sec. 3.1). */
IEWPF_API int iewpf_substeps(iewpf_ctx_t* ctx, int n, double dt);

/* Particle scheme steps (sum over particles of the scheme steps each took)
 * executed by the context so far; one unit of work is a particle scheme
 * step over nx*ny cells (the unit of the throughput metric).
 * Errors: EINVAL, ECUDA. */
IEWPF_API int iewpf_work(iewpf_ctx_t* ctx, int64_t* particle_substeps);

/* Scheme-step kernel of the context (Sec. 3.1; both kinds compute the same
 * scheme, bit for bit).  kind 1: register-marching kernel with nc (2, 3 or
 * 4) columns per lane, `rows` rows per chunk and `warps` (1..8) warps per
 * CTA, using the hardware reciprocal and reciprocal square root; kind 2: the
 * same march with its two Runge-Kutta stages paired in packed f32x2
 * instructions.  Errors: EINVAL (an unknown kind or shape). */
IEWPF_API int iewpf_set_stepper(iewpf_ctx_t* ctx, int kind, int nc, int rows, int warps);

/* Autotuner: times every marching shape on the context's own problem (the
 * state is left unchanged) and keeps the fastest; shape[4] (may be NULL)
 * receives (kind, nc, rows, warps).  Runs by itself before the first
 * forecast unless iewpf_set_stepper was called.  get_stepper reads the
 * current shape.  Errors: EINVAL, ECUDA. */
IEWPF_API int iewpf_tune(iewpf_ctx_t* ctx, int* shape);
IEWPF_API int iewpf_get_stepper(const iewpf_ctx_t* ctx, int* shape);

/* Number of kernels the context has launched so far (a service of the
 * library).  Errors: EINVAL. */
IEWPF_API int iewpf_launch_count(const iewpf_ctx_t* ctx, int64_t* count);

/* ---- batched problems -------------------------------------------- */

/* Many independent assimilation problems of uneven grid and ensemble size
 * advanced together (each with its own parameters, state and observations).
 * Every phase of a cycle (CFL, scheme steps, model error, each analysis step)
 * is one persistent launch over the work of all problems, and the whole
 * forecast-assimilate cycle is one CUDA graph, captured at the first cycle
 * and replayed; the CFL-chosen number of scheme steps per model step drives
 * a conditional while-node of the graph.  Results equal those of the same
 * problems run one by one through iewpf_forecast / iewpf_assimilate. */
typedef struct iewpf_batch iewpf_batch_t;

/* Batched problems (not in the paper, whose experiments run one problem per
 * GPU): n independent IEWPF problems advanced together by persistent
 * kernels, each cycle one CUDA graph.  params[i] as for iewpf_create
 * (n_obs_max >= 1, a distinct instance_id gives independent draws);
 * mooring_xy may be NULL or hold one pointer per problem (NULL for drifter
 * problems).  destroy frees the batch and its contexts (NULL accepted).
 * Errors: EINVAL (n < 1, a problem's parameters), ENOMEM, ECUDA, ENOTPD. */
IEWPF_API int iewpf_batch_create(const iewpf_params_t* params, const double* const* mooring_xy, int n,
                                 iewpf_batch_t** out);
IEWPF_API int iewpf_batch_destroy(iewpf_batch_t* b);

/* The context of problem i (owned by the batch): set or read its state,
 * counters and per-particle diagnostics with the one-problem calls.
 * Errors: EINVAL (i out of range, NULL out). */
IEWPF_API int iewpf_batch_instance(iewpf_batch_t* b, int i, iewpf_ctx_t** ctx);

/* Autotuner of the batched scheme step: shape[4] (may be NULL) receives
 * (kind, columns per lane, rows per chunk, warps per CTA), kind as in
 * iewpf_set_stepper.  Runs by itself before the first cycle.
 * Errors: EINVAL, ECUDA. */
IEWPF_API int iewpf_batch_tune(iewpf_batch_t* b, int* shape);

/* One cycle of every problem: n_model_steps model steps (model error after
 * all but the last, Sec. 4.1) and one IEWPF analysis against obs[i]
 * (obs[i].n_obs must equal problem i's n_obs_max).  diag (may be NULL)
 * receives [n][3] = (w_target, beta, error flags) per problem, w_target
 * being c_bar for the two-stage scheme.  Drifter problems may give their
 * observations as two fixes (value = NULL, see iewpf_obs_t).  Returns the
 * first problem's error, if any: EINVAL (observations that do not fill
 * n_obs_max, non-finite values; refused before any device work), EBETA,
 * EDOMAIN, ENONFINITE, ENOTPD, ECUDA. */
IEWPF_API int iewpf_batch_cycle(iewpf_batch_t* b, int n_model_steps, const iewpf_obs_t* obs, double* diag);

/* A free forecast of every problem (eq. model_equation without
 * assimilation): n_model_steps >= 1 model steps, model error after each when
 * add_model_error, as one CUDA graph (kept for repeated calls with the same
 * arguments).  The states and draw counters advance exactly as n_model_steps
 * steps of iewpf_forecast on each problem would.  Returns the first
 * problem's error (ENONFINITE for a non-finite state), if any. */
IEWPF_API int iewpf_batch_forecast(iewpf_batch_t* b, int n_model_steps, int add_model_error);
IEWPF_API int iewpf_batch_stream(const iewpf_batch_t* b, void** stream);

/* The batch's CUDA stream; the particle scheme steps executed by the batch
 * and the kernel launches it enqueued (a graph replay counts the launches
 * of one capture; either pointer may be NULL); the message of the last
 * error.  Errors: EINVAL, ECUDA. */
IEWPF_API int iewpf_batch_work(iewpf_batch_t* b, int64_t* particle_substeps, int64_t* launches);
IEWPF_API const char* iewpf_batch_last_error(const iewpf_batch_t* b);

/* ------------------------------------------------------------------------
 * Learned surrogate of the forecast model.  The paper forecasts with the
 * numerical scheme only (Sec. 2, Sec. 5.2); this is an addition: a map
 * f_theta: (eta, hu, hv)(t) -> (eta, hu, hv)(t + k dt_model) used in the
 * drift forecast in place of k plain model steps (model error is still added
 * after each of the k steps, from the same Philox streams as the plain path).
 *
 * Network: `depth` periodic 3x3 convolutions, 3 -> width -> ... -> width -> 3
 * channels, SiLU between layers, BF16 weights and activations (NHWC) with
 * FP32 accumulation on the tensor cores; the input is the state times
 * in_scale[c] per field and the output times out_scale[c] is the state
 * change: U(t+k) = U(t) + out_scale * f(in_scale * U(t)).
 * Training loss: mean over pixels and the 3 fields of
 * (f(x) - (Y - X) / out_scale)^2.  Parameters are FP32 masters, flat, per
 * layer l: weights [3][3][cout][cin] (cin padded to 16 for l = 0, cout
 * padded to 16 for the last layer, padding entries zero), then bias[cout].
 * nx and ny must be multiples of 16 and 8.  The object lives on the device
 * current at creation and owns its stream.
 * ------------------------------------------------------------------------ */
typedef struct iewpf_surrogate iewpf_surrogate_t;

/* A network for nx x ny fields: width 64 (or 16), depth >= 2; He-normal
 * weights from `seed`, zero biases, output layer scaled by 0.1 (not in the
 * paper: the learned surrogate described above).  destroy frees it (NULL
 * accepted); param_count gives the length of the flat parameter array.
 * Errors: EINVAL (sizes), ENOMEM, ECUDA. */
IEWPF_API int iewpf_surrogate_create(int nx, int ny, int width, int depth, uint64_t seed, iewpf_surrogate_t** out);
IEWPF_API int iewpf_surrogate_destroy(iewpf_surrogate_t* s);
IEWPF_API int iewpf_surrogate_param_count(const iewpf_surrogate_t* s, int64_t* n);
/* FP32 parameters in the flat layout above (host arrays, copied).
 * Errors: EINVAL (NULL), ECUDA. */
IEWPF_API int iewpf_surrogate_set_params(iewpf_surrogate_t* s, const float* params);
IEWPF_API int iewpf_surrogate_get_params(const iewpf_surrogate_t* s, float* params);
/* Input and output scales per field, in_scale[3], out_scale[3] (> 0, host).
 * Errors: EINVAL (NULL or not positive). */
IEWPF_API int iewpf_surrogate_set_scales(iewpf_surrogate_t* s, const double* in_scale, const double* out_scale);
IEWPF_API int iewpf_surrogate_get_scales(const iewpf_surrogate_t* s, double* in_scale, double* out_scale);
/* Convolution path: 0 (default) = tcgen05 tensor-core kernels where the
 * grid allows, else mma.sync kernels; 1 = always mma.sync.  Inference
 * (apply, the drift forecast) runs on tcgen05 where nx is a multiple of 128
 * and ny even; training (loss_grad, train: the forward pass that keeps the
 * pre-activations, the backward data passes and the weight gradients of
 * layers 1..depth-1) where nx is a multiple of 64 and ny of 4, and an
 * inference on such a grid that the first rule excludes uses the training
 * forward.  The weight gradient of layer 0 (16 input channels) always runs
 * on mma.sync.  get_path writes a bit mask: bit 0 = inference on tcgen05,
 * bit 1 = training on tcgen05.  Errors: EINVAL (path not 0 or 1, NULL). */
IEWPF_API int iewpf_surrogate_set_path(iewpf_surrogate_t* s, int path);
IEWPF_API int iewpf_surrogate_get_path(const iewpf_surrogate_t* s, int* uses_tcgen05);
/* Failure injection for tests of the timeout path (the failure detection
 * of a bounded device wait; no counterpart in the paper).  The next n_evals
 * evaluations of the network on the tcgen05 path (one per chunk of at most
 * 64 fields) run kernels whose CTAs first wait, at most 2^16 polls, on an
 * mbarrier that nothing can complete, before issuing any copy or product;
 * the wait runs out, each CTA records the timeout, frees its tensor memory
 * and exits, so the call returns IEWPF_ETIMEOUT and leaves the context
 * usable.  0 cancels.  The mma.sync path ignores it.
 * Errors: EINVAL (NULL, n_evals < 0). */
IEWPF_API int iewpf_surrogate_inject_timeout(iewpf_surrogate_t* s, int n_evals);
/* U ([n][3][ny][nx] host FP32) -> Unext (same layout), one network call.
 * Errors: EINVAL (n < 1, NULL), ENOMEM, ECUDA, ETIMEOUT (a bounded wait of
 * the tensor-core kernel gave up). */
IEWPF_API int iewpf_surrogate_apply(iewpf_surrogate_t* s, const float* U, int n, float* Unext);
/* The same on device memory: U and Unext (may be equal: in place) are
 * device pointers [n][3][ny][nx], borrowed; the work is ordered after the
 * work queued on `stream` (NULL: the call returns when done) and `stream`
 * waits for it.  Particles go through the network in chunks of 64.  With a
 * stream, a timeout of a bounded wait inside the tensor-core kernel
 * (IEWPF_ETIMEOUT) is reported by the next synchronous call. */
IEWPF_API int iewpf_surrogate_apply_device(iewpf_surrogate_t* s, const float* U, int n, float* Unext, void* stream);
/* The surrogate's own CUDA stream.  Errors: EINVAL. */
IEWPF_API int iewpf_surrogate_stream(const iewpf_surrogate_t* s, void** stream);
/* Loss and its gradient w.r.t. the FP32 parameters (grad[n_params], may be
 * NULL) for the pairs X -> Y ([n][3][ny][nx] host FP32).
 * Errors: EINVAL (n < 1, NULL), ENOMEM, ECUDA. */
IEWPF_API int iewpf_surrogate_loss_grad(iewpf_surrogate_t* s, const float* X, const float* Y, int n, double* loss,
                                        float* grad);
/* Training on n_pairs pairs (psi, M^k psi), M^k = k_steps model steps of the
 * plain stepper of ctx without model error (the deterministic model the
 * surrogate stands for), starting from ctx's state; between two rounds of
 * pairs the ensemble advances k_steps steps with model error (ctx advances).
 * The scales are set from up to 64 pairs spread over the set (unit spread of
 * the input and of the change; one scale for eta, one shared by hu and hv).
 * Then `epochs` shuffled passes of Adam (beta 0.9, 0.999, eps 1e-8, step lr)
 * in mini-batches of `batch` (a last partial batch is skipped);
 * epoch_loss[epochs] (may be NULL) receives the mean batch loss.
 * Errors: EINVAL (sizes that differ from ctx's grid, non-positive counts or
 * rate), ENOMEM, ECUDA, ENONFINITE (a non-finite state while generating
 * the pairs). */
IEWPF_API int iewpf_surrogate_train(iewpf_surrogate_t* s, iewpf_ctx_t* ctx, int n_pairs, int k_steps, int epochs,
                                    int batch, double lr, double* epoch_loss);
/* Device time in seconds of the epochs (the optimizer steps, without the
 * generation of the pairs) of the last successful train call, from CUDA
 * events on the surrogate's stream; 0 before the first.  Errors: EINVAL. */
IEWPF_API int iewpf_surrogate_train_time(const iewpf_surrogate_t* s, double* seconds);
/* Attach (s != NULL, k_steps >= 1) or detach (s = NULL) a surrogate to ctx
 * for drifter_forecast(..., use_surrogate = 1).  Not owned by ctx.  Each
 * surrogate call covers k_steps model steps of all particles; it is rejected
 * and those steps are run by the plain stepper when the network's state is
 * not finite or, for some particle, max|eta| exceeds 1.5 x its value before
 * plus 0.01 m, or the largest |hu/h|, |hv/h| exceeds 1.5 x its value before
 * plus 0.05 m/s.  Errors: EINVAL (k_steps < 1, a network of another grid
 * size). */
IEWPF_API int iewpf_set_surrogate(iewpf_ctx_t* ctx, iewpf_surrogate_t* s, int k_steps);
/* Surrogate calls made for ctx and how many fell back to the plain stepper;
 * the message of a surrogate's last error.  Errors: EINVAL. */
IEWPF_API int iewpf_surrogate_stats(const iewpf_ctx_t* ctx, int64_t* calls, int64_t* fallbacks);
IEWPF_API const char* iewpf_surrogate_last_error(const iewpf_surrogate_t* s);

/* The last factored system (HQH^T + R of Sec. 4.2, eq. S_extended): its
 * order N_y (0 before any factorisation) and the nonzeros of its FP64
 * Cholesky factor strictly below the diagonal (the fill: N_y (N_y - 1) / 2
 * for a dense factor, N_y / 2 for observations that do not interact, whose
 * factor is 2 x 2 blocks).  Synchronises the context's stream.
 * Errors: EINVAL, ECUDA. */
IEWPF_API int iewpf_factor_info(iewpf_ctx_t* ctx, int* n_y, int64_t* nnz_L);

/* Sizes derived from the parameters: the coarse grid Omega^R of Sec. 3.2
 * (nRx x nRy points every c_omega cells) and the pull-stencil radius R;
 * any output pointer may be NULL.  Errors: EINVAL (NULL ctx). */
IEWPF_API int iewpf_sizes(const iewpf_ctx_t* ctx, int* nRx, int* nRy, int* stencil_R);

#ifdef __cplusplus
}
#endif

#endif /* IEWPF_H */
