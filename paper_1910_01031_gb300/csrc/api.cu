// C ABI of the IEWPF library (declared in include/iewpf.h): context
// management, create-time precomputation (pull stencils, SOAR weight table,
// 49x49 block root, mooring factorisation) and the orchestration of the
// forecast and analysis kernels on the context's stream.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/iewpf.h"
#include "common.cuh"
#include "batch.h"
#include "kernels.h"
#include "surrogate.h"
#include <random>

namespace {
// NVTX ranges (domain "iewpf") around each phase of the C ABI, for profilers
// and for filtering a capture to one phase; free when no tool is attached.
nvtxDomainHandle_t nvtx_domain()
{
    static nvtxDomainHandle_t d = nvtxDomainCreateA("iewpf");
    return d;
}

struct Phase {
    explicit Phase(const char* name)
    {
        nvtxEventAttributes_t a = {};
        a.version = NVTX_VERSION;
        a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
        a.messageType = NVTX_MESSAGE_TYPE_ASCII;
        a.message.ascii = name;
        nvtxDomainRangePushEx(nvtx_domain(), &a);
    }
    ~Phase() { nvtxDomainRangePop(nvtx_domain()); }
    Phase(const Phase&) = delete;
    Phase& operator=(const Phase&) = delete;
};
}  // namespace

using namespace iewpf;

struct iewpf_ctx {
    iewpf_params_t P;
    int dev = 0;
    cudaStream_t st = nullptr;
    Grid G{};
    Coarse C{};
    int R = 0;              // pull stencil radius (7 c)
    long long NR = 0;
    long long plane = 0;
    // host precomputations (FP64)
    std::vector<double> K64;   // [2][3][2R+1][2R+1]
    std::vector<double> M49;   // [49][49]
    std::vector<float> wtab;   // [tab][tab]
    // device state
    float* buf[2] = {nullptr, nullptr};
    int* par = nullptr;
    int* nsub = nullptr;
    float* dtp = nullptr;
    float* amax = nullptr;
    int* maxsub = nullptr;
    int* flag = nullptr;
    unsigned long long* work = nullptr;   // particle scheme steps
    float* d_wtab = nullptr;
    float* d_K32 = nullptr;
    double* d_K64 = nullptr;
    float* d_M49 = nullptr;
    // drifters carried by the particles
    double* d_xy = nullptr;
    int nd = 0;
    // analysis buffers
    int nobs_max = 0;
    double* d_obs_xy = nullptr;
    double* d_obs_y = nullptr;
    int* d_cell = nullptr;
    int* d_block0 = nullptr;
    // fixed (mooring) layouts: the local blocks in levels of blocks that share
    // no coarse point (block_levels), applied one level per launch
    int* d_border = nullptr;
    int* d_blevel = nullptr;     // level offsets of d_border (nblev + 1)
    int nblev = 0;
    // fixed layouts of many observations: the factor is that of P A P^T in a
    // nested-dissection order (d_perm_u: unknown i of the factor = unknown
    // d_perm_u[i] of the observations; d_cell_perm: the cells in that order;
    // d_xs: [ne][N_y] solve scratch); null for drifters and small layouts
    int* d_perm_u = nullptr;
    int* d_cell_perm = nullptr;
    double* d_xs = nullptr;
    int ntiles = 0;
    int tile_cap = MAX_TILE_OBS;
    int* d_tile_cnt = nullptr;
    int* d_tile_obs = nullptr;
    double* d_L = nullptr;      // (HQH^T + R) and its factor [Ny][Ny]
    int* d_colptr = nullptr;
    int* d_rowidx = nullptr;
    double* d_rdiag = nullptr;  // 1 / diagonal of the factor [Ny]
    int* d_plan = nullptr;      // level schedule of the triangular sweeps (ana::SolvePlan)
    // a fixed layout's factor values below the diagonal in the order of the
    // plan's rows and of the CSC (launch_pack_factor); null for drifters
    double* d_Lr = nullptr;
    double* d_Lc = nullptr;
    double* d_d = nullptr;      // innovations [ne][Ny]
    double* d_Sd = nullptr;     // [ne][Ny]
    double* d_phi = nullptr;
    double* d_c = nullptr;
    double* d_gamma = nullptr;
    double* d_zeta = nullptr;
    double* d_alpha = nullptr;
    double* d_cstar = nullptr;
    double* d_neglogw = nullptr;
    double* d_coef = nullptr;   // [ne][2] (a_i, length scale)
    double* d_scal = nullptr;   // [4] (c_bar, beta)
    double* d_partial = nullptr;
    int dots_blk = 0;
    float* d_r = nullptr;       // posterior coarse field [ne][N_R]
    float* d_xi = nullptr;      // coarse normals of the model error [ne][N_R]
    float* d_soar = nullptr;    // Q_SOAR^{1/2} of a coarse field [ne][N_R]
    // amax holds the CFL rates of the current state (left there by the last
    // model-error or analysis update); any other change of the state clears it
    bool cfl_ready = false;
    bool factored = false;      // mooring factor ready
    int n_fact = 0;             // order of the last factored HQH^T + R
    // pinned staging
    int* h_flag = nullptr;
    int* h_maxsub = nullptr;
    double* h_scal = nullptr;
    // counters
    uint32_t step = 0, cycle = 0;
    int64_t launches = 0;    // kernels launched
    struct iewpf_surrogate* sur = nullptr;   // learned surrogate for drift forecasts (not owned)
    int sur_k = 0;
    int64_t sur_calls = 0, sur_fallbacks = 0;
    // scheme-step kernel: 1 = register march, 2 = the same with the two stages paired
    int stepper = 1;
    // captured forecasts: device copies of the scheme-step index, the
    // model-step counter and the count of loop iterations, and the graphs
    // by their launch pattern
    int* d_s = nullptr;
    uint32_t* d_step = nullptr;
    unsigned int* d_iters = nullptr;
    uint32_t* h_step = nullptr;
    unsigned int* h_iters = nullptr;
    cudaStream_t st2 = nullptr;
    struct FcGraph {
        int n, err, fixed, have, nd, stepper, nc, TH, warps, paired;
        cudaGraphExec_t exec;
        int64_t launches_fixed, launches_per_iter;
    };
    std::vector<FcGraph> fgraphs;
    MarchShape shape{2, 64, 4};
    bool tuned = false;
    std::string err;
};

namespace {

const char* kNullMsg = "null context";

int fail(iewpf_ctx* c, int code, const std::string& msg)
{
    if (c) c->err = msg;
    return code;
}

#define KL(n, call)                                                                                  \
    do {                                                                                             \
        CK(call);                                                                                    \
        ctx->launches += (n);                                                                        \
    } while (0)

#define CK(call)                                                                                     \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return fail(ctx, IEWPF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));       \
    } while (0)

template <typename T>
int dalloc(iewpf_ctx* ctx, T** p, size_t n)
{
    if (n == 0) n = 1;
    if (cudaMalloc((void**)p, n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, IEWPF_ENOMEM, "device allocation of " + std::to_string(n * sizeof(T)) + " bytes failed");
    }
    return IEWPF_OK;
}

int coarse_count(int n, int c) { return (n - 1 - c / 2) / c + 1; }

// eq. drifterObservation: displacement over dt (minimum image on the
// periodic domain of size Lx by Ly) times H_eq
int drifter_obs_values(double Lx, double Ly, double H, int n, const double* xy, const double* xy_prev, double dt,
                       double* value)
{
    if (n < 0 || (n > 0 && (!xy || !xy_prev || !value)) || !(dt > 0) || !std::isfinite(dt)) return IEWPF_EINVAL;
    const double L[2] = {Lx, Ly};
    for (int k = 0; k < 2 * n; ++k) {
        if (!std::isfinite(xy[k]) || !std::isfinite(xy_prev[k])) return IEWPF_EINVAL;
        const double Lk = L[k & 1];
        double d = std::fmod(xy[k] - xy_prev[k], Lk);
        if (d > 0.5 * Lk) d -= Lk;
        if (d < -0.5 * Lk) d += Lk;
        value[k] = d / dt * H;
    }
    return IEWPF_OK;
}

// the observed values of obs: as given, or formed from the drifters' two
// fixes into tmp; NULL when neither is usable
const double* obs_values(const iewpf_params_t& P, const iewpf_obs_t& o, std::vector<double>& tmp)
{
    if (o.value) return o.value;
    if (P.obs_kind != IEWPF_OBS_DRIFTER || !o.xy || !o.xy_prev) return nullptr;
    tmp.resize(2 * (size_t)std::max(o.n_obs, 0));
    if (drifter_obs_values(P.nx * P.dx, P.ny * P.dy, P.H_eq, o.n_obs, o.xy, o.xy_prev, o.dt, tmp.data()) != IEWPF_OK)
        return nullptr;
    return tmp.data();
}

// every observed value (and position, where given) finite: corrupted
// observations are refused before any device work
bool obs_finite(const iewpf_obs_t& o, const double* value)
{
    for (int k = 0; k < 2 * o.n_obs; ++k)
        if (!std::isfinite(value[k]) || (o.xy && !std::isfinite(o.xy[k]))) return false;
    return true;
}

double soar(double d, double q0, double L0) { return q0 * (1.0 + d / L0) * std::exp(-d / L0); }

// Catmull-Rom weights of taps a-1 .. a+2
void cubic(double t, double w[4])
{
    const double t2 = t * t, t3 = t2 * t;
    w[0] = 0.5 * (-t3 + 2 * t2 - t);
    w[1] = 0.5 * (3 * t3 - 5 * t2 + 2);
    w[2] = 0.5 * (-3 * t3 + 4 * t2 + t);
    w[3] = 0.5 * (t3 - t2);
}

// Response of the chain of eq. detailedOPDUpdate to a unit hu (comp 0) or
// hv (comp 1) observation: point injection on the observation-centred
// coarse lattice, adjoint geostrophic balance with spacing 2 c dx
// (eq. adjointGeoBalance, coefficient g H / f), SOAR twice, bicubic to the
// fine offsets, geostrophic balance on the fine grid.
void build_stencil(const iewpf_params_t& P, int R, std::vector<double>& K)
{
    const int c = P.c_omega, A = 10, n = 2 * A + 1, W = 2 * R + 1, Rf = R + 1, Wf = 2 * Rf + 1;
    const double dxc = c * P.dx, dyc = c * P.dy, s = P.g * P.H_eq / P.f;
    double w5[5][5];
    for (int b = -2; b <= 2; ++b)
        for (int a = -2; a <= 2; ++a) w5[b + 2][a + 2] = soar(std::hypot(a * dxc, b * dyc), P.q0, P.L0);
    K.assign(2 * 3 * W * W, 0.0);
    std::vector<double> e(n * n), t(n * n), eta(Wf * Wf);
    for (int comp = 0; comp < 2; ++comp) {
        std::fill(e.begin(), e.end(), 0.0);
        if (comp == 0) {
            e[(A + 1) * n + A] = -s / (2 * dyc);
            e[(A - 1) * n + A] = s / (2 * dyc);
        } else {
            e[A * n + A + 1] = s / (2 * dxc);
            e[A * n + A - 1] = -s / (2 * dxc);
        }
        for (int pass = 0; pass < 2; ++pass) {
            std::fill(t.begin(), t.end(), 0.0);
            for (int b = 2; b < n - 2; ++b)
                for (int a = 2; a < n - 2; ++a) {
                    double acc = 0.0;
                    for (int db = -2; db <= 2; ++db)
                        for (int da = -2; da <= 2; ++da) acc += w5[db + 2][da + 2] * e[(b + db) * n + a + da];
                    t[b * n + a] = acc;
                }
            e.swap(t);
        }
        for (int fy = -Rf; fy <= Rf; ++fy) {
            const int by = (int)std::floor((double)fy / c);
            double wy[4];
            cubic((double)(fy - by * c) / c, wy);
            for (int fx = -Rf; fx <= Rf; ++fx) {
                const int bx = (int)std::floor((double)fx / c);
                double wx[4];
                cubic((double)(fx - bx * c) / c, wx);
                double acc = 0.0;
                for (int q = 0; q < 4; ++q) {
                    double row = 0.0;
                    for (int p = 0; p < 4; ++p) row += wx[p] * e[(A + by - 1 + q) * n + (A + bx - 1 + p)];
                    acc += wy[q] * row;
                }
                eta[(fy + Rf) * Wf + (fx + Rf)] = acc;
            }
        }
        for (int y = -R; y <= R; ++y)
            for (int x = -R; x <= R; ++x) {
                const int i = (y + Rf) * Wf + (x + Rf);
                const int o = (y + R) * W + (x + R);
                K[(comp * 3 + 0) * W * W + o] = eta[i];
                K[(comp * 3 + 1) * W * W + o] = -s * (eta[i + Wf] - eta[i - Wf]) / (2 * P.dy);
                K[(comp * 3 + 2) * W * W + o] = s * (eta[i + 1] - eta[i - 1]) / (2 * P.dx);
            }
    }
}

// Cyclic Jacobi eigensolver for a symmetric n x n matrix (row-major); on
// return a holds the eigenvalues on its diagonal and v the eigenvectors.
void jacobi_eigen(int n, std::vector<double>& a, std::vector<double>& v)
{
    v.assign(n * n, 0.0);
    for (int i = 0; i < n; ++i) v[i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off += a[i * n + j] * a[i * n + j];
        if (off < 1e-30) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = a[p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                const double th = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
                const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
                const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < n; ++k) {
                    const double akp = a[k * n + p], akq = a[k * n + q];
                    a[k * n + p] = cs * akp - sn * akq;
                    a[k * n + q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < n; ++k) {
                    const double apk = a[p * n + k], aqk = a[q * n + k];
                    a[p * n + k] = cs * apk - sn * aqk;
                    a[q * n + k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = v[k * n + p], vkq = v[k * n + q];
                    v[k * n + p] = cs * vkp - sn * vkq;
                    v[k * n + q] = sn * vkp + cs * vkq;
                }
            }
    }
}

// Square root of the local block I - Q_SOAR Q_GB^T H^T S H Q_GB Q_SOAR of
// eq. svdOfParenthesis on the 7x7 block of a grid with Omega^M = Omega^R
// (spacing c dx).  With B = H Q_GB Q_SOAR (2 x 49) the block is
// I - B^T (B B^T + R)^{-1} B; the root used is V Lambda^{1/2} V^T.
void build_block_root(const iewpf_params_t& P, std::vector<double>& M)
{
    const double dxc = P.c_omega * P.dx, dyc = P.c_omega * P.dy, s = P.g * P.H_eq / P.f;
    auto w = [&](int ax, int ay, int bx, int by) {
        const int dx = ax - bx, dy = ay - by;
        if (std::abs(dx) > 2 || std::abs(dy) > 2) return 0.0;
        return soar(std::hypot(dx * dxc, dy * dyc), P.q0, P.L0);
    };
    double B[2][49];
    for (int m = 0; m < 49; ++m) {
        const int mx = m % 7 - 3, my = m / 7 - 3;
        B[0][m] = -s / (2 * dyc) * (w(0, 1, mx, my) - w(0, -1, mx, my));
        B[1][m] = s / (2 * dxc) * (w(1, 0, mx, my) - w(-1, 0, mx, my));
    }
    double C[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double acc = 0.0;
            for (int m = 0; m < 49; ++m) acc += B[i][m] * B[j][m];
            C[i][j] = acc + (i == j ? P.obs_sigma * P.obs_sigma : 0.0);
        }
    const double det = C[0][0] * C[1][1] - C[0][1] * C[1][0];
    const double S[2][2] = {{C[1][1] / det, -C[0][1] / det}, {-C[1][0] / det, C[0][0] / det}};
    std::vector<double> a(49 * 49), v;
    for (int i = 0; i < 49; ++i)
        for (int j = 0; j < 49; ++j) {
            double acc = 0.0;
            for (int p = 0; p < 2; ++p)
                for (int q = 0; q < 2; ++q) acc += B[p][i] * S[p][q] * B[q][j];
            a[i * 49 + j] = (i == j ? 1.0 : 0.0) - acc;
        }
    for (int i = 0; i < 49; ++i)
        for (int j = i + 1; j < 49; ++j) a[i * 49 + j] = a[j * 49 + i] = 0.5 * (a[i * 49 + j] + a[j * 49 + i]);
    jacobi_eigen(49, a, v);
    M.assign(49 * 49, 0.0);
    for (int k = 0; k < 49; ++k) {
        const double lam = a[k * 49 + k];
        const double sl = lam > 0.0 ? std::sqrt(lam) : 0.0;
        for (int i = 0; i < 49; ++i)
            for (int j = 0; j < 49; ++j) M[i * 49 + j] += v[i * 49 + k] * sl * v[j * 49 + k];
    }
}

cudaError_t launch_step(iewpf_ctx* ctx, int s)
{
    return launch_rk2_march(ctx->buf[0], ctx->buf[1], ctx->par, ctx->nsub, ctx->dtp, s, ctx->G, ctx->shape, ctx->st);
}

// Time every candidate shape of the marching kernel on the context's own
// problem and keep the fastest.  A probe launch reads the current state and
// writes the other buffer without flipping the parity, so the state is left
// as it was; all shapes compute identical values.
int tune_stepper(iewpf_ctx* ctx)
{
    static const int ncs[] = {2, 3, 4};
    static const int ths[] = {16, 32, 64, 128, 256, 512};
    static const int wps[] = {2, 4, 8};
    std::vector<int> ones(ctx->G.ne, 1);
    std::vector<float> dts(ctx->G.ne, (float)(ctx->P.dt_model / 16.0));
    CK(cudaMemcpyAsync(ctx->nsub, ones.data(), sizeof(int) * ones.size(), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->dtp, dts.data(), sizeof(float) * dts.size(), cudaMemcpyHostToDevice, ctx->st));
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    float best = 1e30f;
    MarchShape best_shape = ctx->shape;
    for (int paired = 0; paired < 2; ++paired)
    for (int nc : ncs)
        for (int th : ths) {
            if (th > 2 * ctx->G.ny || (paired && nc == 4)) continue;
            for (int w : wps) {
                MarchShape sh{nc, th, w, paired};
                CK(launch_rk2_march(ctx->buf[0], ctx->buf[1], ctx->par, ctx->nsub, ctx->dtp, 0, ctx->G, sh, ctx->st));
                CK(cudaEventRecord(a, ctx->st));
                for (int r = 0; r < 3; ++r)
                    CK(launch_rk2_march(ctx->buf[0], ctx->buf[1], ctx->par, ctx->nsub, ctx->dtp, 0, ctx->G, sh,
                                        ctx->st));
                CK(cudaEventRecord(b, ctx->st));
                CK(cudaEventSynchronize(b));
                float ms = 0.0f;
                CK(cudaEventElapsedTime(&ms, a, b));
                ctx->launches += 4;
                if (ms < best) {
                    best = ms;
                    best_shape = sh;
                }
            }
        }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->shape = best_shape;
    ctx->stepper = 1 + best_shape.paired;
    ctx->tuned = true;
    return IEWPF_OK;
}

int check_flags(iewpf_ctx* ctx, int f)
{
    if (f & FLAG_NONFINITE) return fail(ctx, IEWPF_ENONFINITE, "non-finite values in the state or weights");
    if (f & FLAG_NOTPD) return fail(ctx, IEWPF_ENOTPD, "HQH^T + R is not positive definite");
    if (f & FLAG_BETA) return fail(ctx, IEWPF_EBETA, "beta < 0: too many observations for the state size");
    if (f & FLAG_DOMAIN) return fail(ctx, IEWPF_EDOMAIN, "alpha solve (Lambert W) out of domain");
    if (f & FLAG_TILE_OVERFLOW) return fail(ctx, IEWPF_EINVAL, "too many observations near one tile");
    if (f & FLAG_TIMEOUT) return fail(ctx, IEWPF_ETIMEOUT, "a bounded wait in a kernel ran out");
    return IEWPF_OK;
}

// Factor (HQH^T + R) for the current d_cell layout.
int factor(iewpf_ctx* ctx, int nobs)
{
    const int n = 2 * nobs;
    KL(1, launch_hqht(ctx->d_K64, ctx->R, ctx->d_cell_perm ? ctx->d_cell_perm : ctx->d_cell, nobs, ctx->G,
                      ctx->P.dense_S,
                   ctx->P.obs_sigma * ctx->P.obs_sigma, ctx->d_L, ctx->st));
    KL(1, launch_cholesky(ctx->d_L, n, ctx->d_colptr, ctx->d_rowidx, ctx->flag, ctx->d_rdiag, ctx->d_plan, ctx->st));
    ctx->n_fact = n;
    return IEWPF_OK;
}

int upload_obs_layout(iewpf_ctx* ctx, const double* xy, int nobs)
{
    CK(cudaMemcpyAsync(ctx->d_obs_xy, xy, sizeof(double) * 2 * nobs, cudaMemcpyHostToDevice, ctx->st));
    KL(2, launch_obs_setup(ctx->d_obs_xy, nobs, ctx->G, ctx->C, ctx->P.dx, ctx->P.dy, ctx->R, ctx->d_cell,
                        ctx->d_block0, ctx->d_tile_cnt, ctx->d_tile_obs, ctx->tile_cap, ctx->flag, ctx->st));
    return IEWPF_OK;
}

int read_flags(iewpf_ctx* ctx)
{
    CK(cudaMemcpyAsync(ctx->h_flag, ctx->flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    const int f = *ctx->h_flag;
    if (f) {
        CK(cudaMemsetAsync(ctx->flag, 0, sizeof(int), ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
    }
    return check_flags(ctx, f);
}

// Captures n_steps model steps into one executable graph: per model step the
// CFL pass, a conditional WHILE node whose body is one scheme step (with the
// drifters) and the loop control reading the largest n_sub on the device, the
// parity flip, and the model error.  The scheme-step index and the model-step
// counter come from device memory, so the graph serves every call with the
// same pattern and needs no host synchronisation between model steps.
static cudaError_t capture_forecast(iewpf_ctx* ctx, int n_steps, int add_err, int fixed, bool have0,
                                    iewpf_ctx::FcGraph& fg)
{
    cudaStream_t st = ctx->st, st2 = ctx->st2;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    int64_t fixed_launches = 0;
    const int64_t per_iter = 2 + (ctx->nd > 0 ? 1 : 0);
    bool have = have0;
    auto body = [&]() -> cudaError_t {
        cudaError_t r;
        for (int k = 0; k < n_steps; ++k) {
            if ((r = launch_cfl(ctx->buf[0], ctx->buf[1], ctx->par, ctx->amax, ctx->nsub, ctx->dtp, ctx->maxsub,
                                ctx->G, ctx->P.courant, ctx->P.dt_model, fixed, st, have, ctx->flag)) != cudaSuccess)
                return r;
            fixed_launches += (fixed > 0 || have) ? 1 : 2;
            if ((r = launch_step_reset(ctx->d_s, st)) != cudaSuccess) return r;
            fixed_launches += 1;
            cudaStreamCaptureStatus status;
            cudaGraph_t g = nullptr;
            const cudaGraphNode_t* deps = nullptr;
            size_t ndeps = 0;
            if ((r = cudaStreamGetCaptureInfo(st, &status, nullptr, &g, &deps, nullptr, &ndeps)) != cudaSuccess)
                return r;
            cudaGraphConditionalHandle h;
            if ((r = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess) return r;
            cudaGraphNodeParams prm = {};
            prm.type = cudaGraphNodeTypeConditional;
            prm.conditional.handle = h;
            prm.conditional.type = cudaGraphCondTypeWhile;
            prm.conditional.size = 1;
            cudaGraphNode_t node;
            if ((r = cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &prm)) != cudaSuccess) return r;
            cudaGraph_t loop = prm.conditional.phGraph_out[0];
            if ((r = cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
                cudaSuccess)
                return r;
            if ((r = cudaStreamBeginCaptureToGraph(st2, loop, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
                cudaSuccess)
                return r;
            cudaError_t rb = launch_rk2_march(ctx->buf[0], ctx->buf[1], ctx->par, ctx->nsub, ctx->dtp, 0, ctx->G,
                                              ctx->shape, st2, ctx->d_s);
            if (rb == cudaSuccess && ctx->nd > 0)
                rb = launch_drift(ctx->buf[0], ctx->buf[1], ctx->par, ctx->nsub, ctx->dtp, ctx->d_xy, ctx->nd, 0,
                                  ctx->G, ctx->P.dx, ctx->P.dy, st2, ctx->d_s);
            if (rb == cudaSuccess) rb = launch_step_ctl(ctx->d_s, ctx->maxsub, h, ctx->d_iters, st2);
            r = cudaStreamEndCapture(st2, &loop);
            if (rb != cudaSuccess) return rb;
            if (r != cudaSuccess) return r;
            if ((r = launch_par_update(ctx->par, ctx->nsub, ctx->G.ne, ctx->work, st)) != cudaSuccess) return r;
            fixed_launches += 1;
            if (add_err) {
                QhalfArgs A{};
                A.b0 = ctx->buf[0];
                A.b1 = ctx->buf[1];
                A.par = ctx->par;
                A.wtab = ctx->d_wtab;
                A.from_philox = 1;
                A.seed = ctx->P.seed;
                A.t = 0;
                A.t_dev = ctx->d_step;
                A.stream = 0u + 16u * (uint32_t)ctx->P.instance_id;
                A.xi_buf = ctx->d_xi;
                A.soar_buf = ctx->d_soar;
                A.amax = ctx->amax;
                if ((r = cudaMemsetAsync(ctx->amax, 0, sizeof(float) * ctx->G.ne, st)) != cudaSuccess) return r;
                if ((r = launch_qhalf(A, ctx->G, ctx->C, st)) != cudaSuccess) return r;
                fixed_launches += qhalf_launches(A);
            }
            have = add_err && fixed <= 0;
            if ((r = launch_counter_inc(ctx->d_step, st)) != cudaSuccess) return r;
            fixed_launches += 1;
        }
        return cudaSuccess;
    };
    cudaError_t eb = body();
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(st, &graph);
    if (eb == cudaSuccess) eb = e;
    if (eb == cudaSuccess) eb = cudaGraphInstantiate(&fg.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    fg.launches_fixed = fixed_launches;
    fg.launches_per_iter = per_iter;
    return eb;
}

int forecast_impl(iewpf_ctx* ctx, int n_steps, int add_err, int fixed)
{
    if (!ctx) return IEWPF_EINVAL;
    if (n_steps < 0) return fail(ctx, IEWPF_EINVAL, "n_model_steps < 0");
    CK(cudaSetDevice(ctx->dev));
    int rc;
    if (!ctx->tuned && (rc = tune_stepper(ctx))) return rc;
    if (n_steps > 0) {
        const int have = ctx->cfl_ready && fixed <= 0;
        iewpf_ctx::FcGraph key{n_steps, add_err ? 1 : 0, fixed, have, ctx->nd, ctx->stepper, ctx->shape.nc,
                               ctx->shape.TH, ctx->shape.warps, ctx->shape.paired, nullptr, 0, 0};
        iewpf_ctx::FcGraph* fg = nullptr;
        for (auto& g : ctx->fgraphs)
            if (g.n == key.n && g.err == key.err && g.fixed == key.fixed && g.have == key.have && g.nd == key.nd &&
                g.stepper == key.stepper && g.nc == key.nc && g.TH == key.TH && g.warps == key.warps &&
                g.paired == key.paired)
                fg = &g;
        if (!fg) {
            if (ctx->fgraphs.size() >= 8) {
                cudaGraphExecDestroy(ctx->fgraphs.front().exec);
                ctx->fgraphs.erase(ctx->fgraphs.begin());
            }
            CK(capture_forecast(ctx, n_steps, add_err, fixed, have != 0, key));
            ctx->fgraphs.push_back(key);
            fg = &ctx->fgraphs.back();
        }
        *ctx->h_step = ctx->step;
        CK(cudaMemcpyAsync(ctx->d_step, ctx->h_step, sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->st));
        CK(cudaMemsetAsync(ctx->d_iters, 0, sizeof(unsigned int), ctx->st));
        CK(cudaGraphLaunch(fg->exec, ctx->st));
        CK(cudaMemcpyAsync(ctx->h_iters, ctx->d_iters, sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->st));
        ctx->launches += fg->launches_fixed;
        ctx->step += (uint32_t)n_steps;
        ctx->cfl_ready = add_err && fixed <= 0;
    }
    KL(1, launch_nonfinite(ctx->buf[0], ctx->buf[1], ctx->par, ctx->G, ctx->flag, ctx->st));
    rc = read_flags(ctx);
    if (n_steps > 0) ctx->launches += (int64_t)*ctx->h_iters * (2 + (ctx->nd > 0 ? 1 : 0));
    return rc;
}

}  // namespace

struct iewpf_surrogate {
    Surrogate net;
    cudaStream_t st = nullptr;
    int dev = 0;
    std::string err;
    // inference scratch of an attached context
    float* S0 = nullptr;
    float* S1 = nullptr;
    float* stats = nullptr;
    size_t cap_state = 0;
    int chunk = 64;
    double train_s = 0.0;       // device time of the epochs of the last train call
};

// the timeout flag of the network's tensor-core kernels (read and cleared)
static int sur_flag(iewpf_surrogate* s, cudaStream_t st)
{
    int f = 0;
    if (cudaMemcpyAsync(&f, s->net.dflag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        s->err = "reading the kernel flag";
        return IEWPF_ECUDA;
    }
    if (f) {
        cudaMemsetAsync(s->net.dflag, 0, sizeof(int), st);
        cudaStreamSynchronize(st);
        s->err = "a bounded wait of the tensor-core convolution ran out";
        return IEWPF_ETIMEOUT;
    }
    return IEWPF_OK;
}

namespace {

// k model steps of every particle by the surrogate (in place of k steps of
// the scheme of Sec. 2 in the drift forecast of Sec. 5.2): the state change
// of k steps from the network, drifters advected with the mean of the
// velocities before and after, then the k model errors of those steps.  The
// plain scheme takes over for the k steps when the network's state fails the
// guard: non-finite, or for some particle max|eta| or the largest velocity
// component grows by more than SUR_GROWTH (plus a small absolute slack).
constexpr float SUR_GROWTH = 1.5f, SUR_SLACK_ETA = 0.01f, SUR_SLACK_VEL = 0.05f;

int surrogate_steps(iewpf_ctx* ctx)
{
    iewpf_surrogate* S = ctx->sur;
    const int ne = ctx->G.ne, k = ctx->sur_k;
    const size_t nstate = (size_t)ne * 3 * ctx->plane;
    CK(cudaSetDevice(ctx->dev));
    if (S->cap_state < nstate) {
        if (S->S0) cudaFree(S->S0);
        if (S->S1) cudaFree(S->S1);
        if (S->stats) cudaFree(S->stats);
        S->S0 = S->S1 = nullptr;
        S->stats = nullptr;
        S->cap_state = 0;
        if (cudaMalloc((void**)&S->S0, nstate * 4) != cudaSuccess || cudaMalloc((void**)&S->S1, nstate * 4) != cudaSuccess ||
            cudaMalloc((void**)&S->stats, sizeof(float) * 4 * ne) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, IEWPF_ENOMEM, "surrogate scratch");
        }
        S->cap_state = nstate;
    }
    int rc;
    if ((rc = iewpf_get_state(ctx, S->S0, 1, nullptr))) return rc;
    CK(cudaMemcpyAsync(S->S1, S->S0, nstate * 4, cudaMemcpyDeviceToDevice, ctx->st));
    const size_t per = 3 * (size_t)ctx->plane;
    for (int p0 = 0; p0 < ne; p0 += S->chunk) {
        const int nb = std::min(S->chunk, ne - p0);
        if ((rc = S->net.infer(S->S0 + per * p0, nb, ctx->st))) return fail(ctx, rc, "surrogate network");
        CK(S->net.apply(S->S1 + per * p0, nb, ctx->st));
        ctx->launches += 2 + S->net.depth;
    }
    // guard: per-particle max|eta| and max velocity component before / after
    KL(1, launch_sur_stats(S->S0, ne, ctx->G, S->stats, ctx->st));
    KL(1, launch_sur_stats(S->S1, ne, ctx->G, S->stats + 2 * ne, ctx->st));
    std::vector<float> st(4 * (size_t)ne);
    CK(cudaMemcpyAsync(st.data(), S->stats, sizeof(float) * 4 * ne, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if ((rc = sur_flag(S, ctx->st))) return fail(ctx, rc, S->err);
    ctx->sur_calls++;
    bool ok = true;
    for (int p = 0; p < ne && ok; ++p) {
        const float e0 = st[2 * p], v0 = st[2 * p + 1], e1 = st[2 * ne + 2 * p], v1 = st[2 * ne + 2 * p + 1];
        ok = std::isfinite(e1) && std::isfinite(v1) && e1 <= SUR_GROWTH * e0 + SUR_SLACK_ETA &&
             v1 <= SUR_GROWTH * v0 + SUR_SLACK_VEL;
    }
    if (!ok) {
        ctx->sur_fallbacks++;
        return forecast_impl(ctx, k, 1, 0);
    }
    if (ctx->nd > 0)
        KL(1, launch_sur_drift(S->S0, S->S1, ne, ctx->nd, ctx->d_xy, ctx->G, ctx->P.dx, ctx->P.dy,
                               k * ctx->P.dt_model, ctx->st));
    if ((rc = iewpf_set_state(ctx, S->S1, 1, nullptr))) return rc;
    for (int i = 0; i < k; ++i) {
        QhalfArgs A{};
        A.b0 = ctx->buf[0];
        A.b1 = ctx->buf[1];
        A.par = ctx->par;
        A.wtab = ctx->d_wtab;
        A.from_philox = 1;
        A.seed = ctx->P.seed;
        A.t = ctx->step + i;
        A.t_dev = nullptr;
        A.stream = 16u * (uint32_t)ctx->P.instance_id;
        A.xi_buf = ctx->d_xi;
        A.soar_buf = ctx->d_soar;
        KL(qhalf_launches(A), launch_qhalf(A, ctx->G, ctx->C, ctx->st));
    }
    ctx->step += k;
    KL(1, launch_nonfinite(ctx->buf[0], ctx->buf[1], ctx->par, ctx->G, ctx->flag, ctx->st));
    return read_flags(ctx);
}

}  // namespace

extern "C" {

int iewpf_create(const iewpf_params_t* params, const double* mooring_xy, iewpf_ctx_t** out)
{
    Phase phase_("create");
    if (!params || !out) return IEWPF_EINVAL;
    *out = nullptr;
    const iewpf_params_t& P = *params;
    const int c = P.c_omega;
    if (c < 1 || c % 2 == 0 || c > 15 || P.nx <= 14 * c + 1 || P.ny <= 14 * c + 1 || !(P.dx > 0) ||
        !(P.dy > 0) || !(P.H_eq > 0) || !(P.g > 0) || P.f == 0.0 || !(P.dt_model > 0) || !(P.courant > 0) ||
        !(P.q0 >= 0) || !(P.L0 > 0) || P.n_particles < 1 || P.n_particles > 65535 || P.n_obs_max < 0 ||
        !(P.obs_sigma > 0) || P.theta < 1.0 || P.theta > 2.0 || P.n_drifters_max < 0 ||
        (P.obs_kind != IEWPF_OBS_DRIFTER && P.obs_kind != IEWPF_OBS_MOORING) ||
        (P.obs_kind == IEWPF_OBS_MOORING && P.n_obs_max > 0 && !mooring_xy) || P.instance_id < 0 ||
        P.instance_id > 0x0FFFFFFF || (P.scheme != IEWPF_TWO_STAGE && P.scheme != IEWPF_ONE_STAGE))
        return IEWPF_EINVAL;
    iewpf_ctx* ctx = new (std::nothrow) iewpf_ctx();
    if (!ctx) return IEWPF_ENOMEM;
    ctx->P = P;
    auto bail = [&](int code) {
        iewpf_destroy(ctx);
        return code;
    };
    if (cudaGetDevice(&ctx->dev) != cudaSuccess) return bail(IEWPF_ECUDA);
    if (cudaStreamCreateWithFlags(&ctx->st, cudaStreamNonBlocking) != cudaSuccess) return bail(IEWPF_ECUDA);
    Grid& G = ctx->G;
    G.nx = P.nx;
    G.ny = P.ny;
    G.dx = (float)P.dx;
    G.dy = (float)P.dy;
    G.g = (float)P.g;
    G.f = (float)P.f;
    G.H = (float)P.H_eq;
    G.theta = (float)P.theta;
    G.inv_dx = (float)(1.0 / P.dx);
    G.inv_dy = (float)(1.0 / P.dy);
    G.fdx = (float)(P.f * P.dx);
    G.fdy = (float)(P.f * P.dy);
    G.fdx_half = (float)(0.5 * P.f * P.dx);
    G.fdy_half = (float)(0.5 * P.f * P.dy);
    G.inv_2g = (float)(0.5 / P.g);
    G.sgh = (float)(P.g * P.H_eq / P.f);
    G.inv_2dx = (float)(0.5 / P.dx);
    G.inv_2dy = (float)(0.5 / P.dy);
    G.theta2 = 2.0f * G.theta;
    G.fdx2 = 2.0f * G.fdx;
    G.fdy2 = 2.0f * G.fdy;
    G.inv_4g = 0.5f * G.inv_2g;
    G.g_half = 0.5f * G.g;
    G.gH = (float)(P.g * P.H_eq);
    G.ne = P.n_particles;
    G.plane = (long long)P.nx * P.ny;
    ctx->plane = G.plane;
    Coarse& C = ctx->C;
    C.c = c;
    C.o = c / 2;
    C.nRx = coarse_count(P.nx, c);
    C.nRy = coarse_count(P.ny, c);
    C.tab = 3 * c;
    ctx->NR = (long long)C.nRx * C.nRy;
    ctx->R = 7 * c;
    // SOAR weights by fine-cell offset
    ctx->wtab.resize(C.tab * C.tab);
    for (int y = 0; y < C.tab; ++y)
        for (int x = 0; x < C.tab; ++x)
            ctx->wtab[y * C.tab + x] = (float)soar(std::hypot(x * P.dx, y * P.dy), P.q0, P.L0);
    build_stencil(P, ctx->R, ctx->K64);
    build_block_root(P, ctx->M49);
    const size_t ne = P.n_particles;
    const size_t state = ne * 3 * (size_t)G.plane;
    int rc;
    if ((rc = dalloc(ctx, &ctx->buf[0], state)) || (rc = dalloc(ctx, &ctx->buf[1], state)) ||
        (rc = dalloc(ctx, &ctx->par, ne)) || (rc = dalloc(ctx, &ctx->nsub, ne)) ||
        (rc = dalloc(ctx, &ctx->dtp, ne)) || (rc = dalloc(ctx, &ctx->amax, ne)) ||
        (rc = dalloc(ctx, &ctx->maxsub, 1)) || (rc = dalloc(ctx, &ctx->flag, 1)) || (rc = dalloc(ctx, &ctx->work, 1)) ||
        (rc = dalloc(ctx, &ctx->d_wtab, ctx->wtab.size())) || (rc = dalloc(ctx, &ctx->d_K32, ctx->K64.size())) ||
        (rc = dalloc(ctx, &ctx->d_K64, ctx->K64.size())) || (rc = dalloc(ctx, &ctx->d_M49, 49 * 49)))
        return bail(rc);
    if (cudaMallocHost((void**)&ctx->h_flag, sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void**)&ctx->h_maxsub, sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void**)&ctx->h_scal, 4 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void**)&ctx->h_step, sizeof(uint32_t)) != cudaSuccess ||
        cudaMallocHost((void**)&ctx->h_iters, sizeof(unsigned int)) != cudaSuccess)
        return bail(IEWPF_ENOMEM);
    if ((rc = dalloc(ctx, &ctx->d_s, 1)) || (rc = dalloc(ctx, &ctx->d_step, 1)) || (rc = dalloc(ctx, &ctx->d_iters, 1)))
        return bail(rc);
    if (cudaStreamCreateWithFlags(&ctx->st2, cudaStreamNonBlocking) != cudaSuccess) return bail(IEWPF_ECUDA);
    std::vector<float> K32(ctx->K64.begin(), ctx->K64.end());
    std::vector<float> M32(ctx->M49.begin(), ctx->M49.end());
    if (cudaMemsetAsync(ctx->buf[0], 0, state * sizeof(float), ctx->st) != cudaSuccess ||
        cudaMemsetAsync(ctx->buf[1], 0, state * sizeof(float), ctx->st) != cudaSuccess ||
        cudaMemsetAsync(ctx->par, 0, ne * sizeof(int), ctx->st) != cudaSuccess ||
        cudaMemsetAsync(ctx->flag, 0, sizeof(int), ctx->st) != cudaSuccess ||
        cudaMemsetAsync(ctx->work, 0, sizeof(unsigned long long), ctx->st) != cudaSuccess ||
        cudaMemcpyAsync(ctx->d_wtab, ctx->wtab.data(), ctx->wtab.size() * 4, cudaMemcpyHostToDevice, ctx->st) ||
        cudaMemcpyAsync(ctx->d_K32, K32.data(), K32.size() * 4, cudaMemcpyHostToDevice, ctx->st) ||
        cudaMemcpyAsync(ctx->d_K64, ctx->K64.data(), ctx->K64.size() * 8, cudaMemcpyHostToDevice, ctx->st) ||
        cudaMemcpyAsync(ctx->d_M49, M32.data(), M32.size() * 4, cudaMemcpyHostToDevice, ctx->st) ||
        cudaStreamSynchronize(ctx->st) != cudaSuccess)
        return bail(IEWPF_ECUDA);
    // analysis buffers
    const int nobs = P.n_obs_max;
    ctx->nobs_max = nobs;
    const size_t ny = 2 * (size_t)std::max(nobs, 1);
    ctx->ntiles = ((P.nx + OBS_TX - 1) / OBS_TX) * ((P.ny + OBS_TY - 1) / OBS_TY);
    ctx->dots_blk = rand_dots_blocks((int)ctx->NR);
    if ((rc = dalloc(ctx, &ctx->d_obs_xy, ny)) || (rc = dalloc(ctx, &ctx->d_obs_y, ny)) ||
        (rc = dalloc(ctx, &ctx->d_cell, ny)) || (rc = dalloc(ctx, &ctx->d_block0, ny)) ||
        (rc = dalloc(ctx, &ctx->d_tile_cnt, ctx->ntiles)) ||
        (rc = dalloc(ctx, &ctx->d_tile_obs, (size_t)ctx->ntiles * ctx->tile_cap)) ||
        (rc = dalloc(ctx, &ctx->d_L, ny * ny)) || (rc = dalloc(ctx, &ctx->d_colptr, ny + 1)) ||
        (rc = dalloc(ctx, &ctx->d_rowidx, ny * (ny - 1) / 2 + ny)) || (rc = dalloc(ctx, &ctx->d_d, ne * ny)) ||
        (rc = dalloc(ctx, &ctx->d_rdiag, ny)) || (rc = dalloc(ctx, &ctx->d_plan, solve_plan_ints((int)ny))) ||
        (rc = dalloc(ctx, &ctx->d_Sd, ne * ny)) || (rc = dalloc(ctx, &ctx->d_phi, ne)) ||
        (rc = dalloc(ctx, &ctx->d_c, ne)) || (rc = dalloc(ctx, &ctx->d_gamma, ne)) ||
        (rc = dalloc(ctx, &ctx->d_zeta, ne)) || (rc = dalloc(ctx, &ctx->d_alpha, ne)) ||
        (rc = dalloc(ctx, &ctx->d_cstar, ne)) || (rc = dalloc(ctx, &ctx->d_neglogw, ne)) ||
        (rc = dalloc(ctx, &ctx->d_coef, 2 * ne)) || (rc = dalloc(ctx, &ctx->d_scal, 4)) ||
        (rc = dalloc(ctx, &ctx->d_partial, ne * ctx->dots_blk * 3)) ||
        (rc = dalloc(ctx, &ctx->d_r, ne * (size_t)ctx->NR)) || (rc = dalloc(ctx, &ctx->d_xi, ne * (size_t)ctx->NR)) ||
        (rc = dalloc(ctx, &ctx->d_soar, ne * (size_t)ctx->NR)))
        return bail(rc);
    if (P.n_drifters_max > 0 && (rc = dalloc(ctx, &ctx->d_xy, ne * 2 * (size_t)P.n_drifters_max)))
        return bail(rc);
    if (P.obs_kind == IEWPF_OBS_MOORING && nobs > 0) {
        if ((rc = upload_obs_layout(ctx, mooring_xy, nobs))) return bail(rc);
        if (nobs >= kNdMinObs) {
            // many fixed observations: factor in a nested-dissection order of
            // their coupling graph (wide levels for the triangular sweeps)
            std::vector<int> cells(2 * (size_t)nobs), order;
            if (cudaMemcpy(cells.data(), ctx->d_cell, sizeof(int) * 2 * nobs, cudaMemcpyDeviceToHost) != cudaSuccess)
                return bail(IEWPF_ECUDA);
            // (no coupled pair: the factor is 2 x 2 blocks in any order)
            const bool coupled = nd_order(cells.data(), nobs, ctx->G.nx, ctx->G.ny, ctx->R, order) > 0;
            std::vector<int> perm_u(2 * (size_t)nobs), cells_p(2 * (size_t)nobs);
            for (int i = 0; i < nobs; ++i) {
                perm_u[2 * i] = 2 * order[i];
                perm_u[2 * i + 1] = 2 * order[i] + 1;
                cells_p[2 * i] = cells[2 * order[i]];
                cells_p[2 * i + 1] = cells[2 * order[i] + 1];
            }
            if (coupled && ((rc = dalloc(ctx, &ctx->d_perm_u, 2 * (size_t)nobs)) ||
                            (rc = dalloc(ctx, &ctx->d_cell_perm, 2 * (size_t)nobs)) ||
                            (rc = dalloc(ctx, &ctx->d_xs, (size_t)ne * 2 * nobs))))
                return bail(rc);
            if (coupled &&
                (cudaMemcpy(ctx->d_perm_u, perm_u.data(), sizeof(int) * 2 * nobs, cudaMemcpyHostToDevice) !=
                     cudaSuccess ||
                 cudaMemcpy(ctx->d_cell_perm, cells_p.data(), sizeof(int) * 2 * nobs, cudaMemcpyHostToDevice) !=
                     cudaSuccess))
                return bail(IEWPF_ECUDA);
        }
        if ((rc = factor(ctx, nobs)) || (rc = read_flags(ctx))) return bail(rc);
        // the factor's non-zeros below the diagonal (the stream is idle after read_flags)
        int nnz = 0;
        if (cudaMemcpy(&nnz, ctx->d_colptr + 2 * nobs, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return bail(IEWPF_ECUDA);
        if ((rc = dalloc(ctx, &ctx->d_Lr, (size_t)nnz)) || (rc = dalloc(ctx, &ctx->d_Lc, (size_t)nnz))) return bail(rc);
        if (launch_pack_factor(ctx->d_L, 2 * nobs, ctx->d_colptr, ctx->d_rowidx, ctx->d_plan, ctx->d_Lr, ctx->d_Lc,
                               ctx->st) != cudaSuccess)
            return bail(IEWPF_ECUDA);
        ctx->factored = true;
        // levels of the local blocks of the fixed layout
        std::vector<int> b0(2 * (size_t)nobs), order;
        if (cudaMemcpy(b0.data(), ctx->d_block0, sizeof(int) * 2 * nobs, cudaMemcpyDeviceToHost) != cudaSuccess)
            return bail(IEWPF_ECUDA);
        std::vector<int> level_off;
        block_levels(b0.data(), nobs, ctx->C.nRx, ctx->C.nRy, order, level_off);
        ctx->nblev = (int)level_off.size() - 1;
        if ((rc = dalloc(ctx, &ctx->d_border, nobs)) || (rc = dalloc(ctx, &ctx->d_blevel, level_off.size())) ||
            cudaMemcpy(ctx->d_border, order.data(), sizeof(int) * nobs, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(ctx->d_blevel, level_off.data(), sizeof(int) * level_off.size(), cudaMemcpyHostToDevice) !=
                cudaSuccess)
            return bail(rc ? rc : IEWPF_ECUDA);
    }
    *out = ctx;
    return IEWPF_OK;
}

int iewpf_destroy(iewpf_ctx_t* ctx)
{
    if (!ctx) return IEWPF_OK;
    cudaSetDevice(ctx->dev);
    if (ctx->st) cudaStreamSynchronize(ctx->st);
    void* ptrs[] = {ctx->buf[0], ctx->buf[1], ctx->par, ctx->nsub, ctx->dtp, ctx->amax, ctx->maxsub, ctx->flag, ctx->work,
                    ctx->d_wtab, ctx->d_K32, ctx->d_K64, ctx->d_M49, ctx->d_xy, ctx->d_obs_xy, ctx->d_obs_y,
                    ctx->d_cell, ctx->d_block0, ctx->d_border, ctx->d_blevel, ctx->d_perm_u, ctx->d_cell_perm, ctx->d_xs,
                    ctx->d_tile_cnt, ctx->d_tile_obs, ctx->d_L, ctx->d_colptr,
                    ctx->d_rowidx, ctx->d_rdiag, ctx->d_plan, ctx->d_Lr, ctx->d_Lc, ctx->d_d, ctx->d_Sd, ctx->d_phi, ctx->d_c, ctx->d_gamma, ctx->d_zeta,
                    ctx->d_alpha, ctx->d_cstar, ctx->d_neglogw, ctx->d_coef, ctx->d_scal, ctx->d_partial,
                    ctx->d_r, ctx->d_xi, ctx->d_soar};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (ctx->h_flag) cudaFreeHost(ctx->h_flag);
    if (ctx->h_maxsub) cudaFreeHost(ctx->h_maxsub);
    if (ctx->h_scal) cudaFreeHost(ctx->h_scal);
    if (ctx->h_step) cudaFreeHost(ctx->h_step);
    if (ctx->h_iters) cudaFreeHost(ctx->h_iters);
    for (auto& fg : ctx->fgraphs) cudaGraphExecDestroy(fg.exec);
    for (void* p : {(void*)ctx->d_s, (void*)ctx->d_step, (void*)ctx->d_iters})
        if (p) cudaFree(p);
    if (ctx->st2) cudaStreamDestroy(ctx->st2);
    if (ctx->st) cudaStreamDestroy(ctx->st);
    delete ctx;
    return IEWPF_OK;
}

static int copy_state(iewpf_ctx_t* ctx, float* host_or_dev, int on_device, void* stream, bool in)
{
    if (!ctx) return IEWPF_EINVAL;
    if (in) ctx->cfl_ready = false;
    if (!host_or_dev) return fail(ctx, IEWPF_EINVAL, "null state pointer");
    CK(cudaSetDevice(ctx->dev));
    cudaStream_t user = (cudaStream_t)stream;
    if (user) {
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CK(cudaEventRecord(ev, user));
        CK(cudaStreamWaitEvent(ctx->st, ev, 0));
        CK(cudaEventDestroy(ev));
    }
    const size_t per = 3 * (size_t)ctx->plane;
    std::vector<int> par(ctx->G.ne);
    if (!in) {
        CK(cudaMemcpyAsync(par.data(), ctx->par, sizeof(int) * par.size(), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
    }
    const cudaMemcpyKind kind = in ? (on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice)
                                   : (on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
    if (in) {
        CK(cudaMemcpyAsync(ctx->buf[0], host_or_dev, sizeof(float) * per * ctx->G.ne, kind, ctx->st));
        CK(cudaMemsetAsync(ctx->par, 0, sizeof(int) * ctx->G.ne, ctx->st));
    } else {
        // contiguous runs of particles that live in the same buffer
        int p = 0;
        while (p < ctx->G.ne) {
            int q = p;
            while (q < ctx->G.ne && par[q] == par[p]) ++q;
            CK(cudaMemcpyAsync(host_or_dev + per * p, ctx->buf[par[p]] + per * p, sizeof(float) * per * (q - p),
                               kind, ctx->st));
            p = q;
        }
    }
    CK(cudaStreamSynchronize(ctx->st));
    return IEWPF_OK;
}

int iewpf_set_state(iewpf_ctx_t* ctx, const float* src, int on_device, void* stream)
{
    return copy_state(ctx, const_cast<float*>(src), on_device, stream, true);
}

int iewpf_get_state(iewpf_ctx_t* ctx, float* dst, int on_device, void* stream)
{
    return copy_state(ctx, dst, on_device, stream, false);
}

int iewpf_forecast(iewpf_ctx_t* ctx, int n_model_steps, int add_model_error)
{
    Phase phase_("forecast");
    return forecast_impl(ctx, n_model_steps, add_model_error, 0);
}

int iewpf_forecast_fixed(iewpf_ctx_t* ctx, int n_model_steps, int add_model_error, int n_sub)
{
    Phase phase_("forecast");
    if (!ctx) return IEWPF_EINVAL;
    if (n_sub < 1) return fail(ctx, IEWPF_EINVAL, "n_sub < 1");
    return forecast_impl(ctx, n_model_steps, add_model_error, n_sub);
}

int iewpf_assimilate(iewpf_ctx_t* ctx, const iewpf_obs_t* obs, iewpf_diag_t* diag)
{
    Phase phase_("assimilate");
    if (!ctx) return IEWPF_EINVAL;
    if (!obs || obs->n_obs < 1 || obs->n_obs > ctx->nobs_max) return fail(ctx, IEWPF_EINVAL, "bad observation set");
    const bool mooring = ctx->P.obs_kind == IEWPF_OBS_MOORING;
    if (!mooring && !obs->xy) return fail(ctx, IEWPF_EINVAL, "drifter observations need positions");
    if (mooring && obs->n_obs != ctx->nobs_max)
        return fail(ctx, IEWPF_EINVAL, "mooring observations must cover every mooring");
    std::vector<double> derived;
    const double* value = obs_values(ctx->P, *obs, derived);
    if (!value) return fail(ctx, IEWPF_EINVAL, "no observed values (and no usable previous drifter fixes)");
    if (!obs_finite(*obs, value)) return fail(ctx, IEWPF_EINVAL, "non-finite observation value or position");
    CK(cudaSetDevice(ctx->dev));
    const int nobs = obs->n_obs, n = 2 * nobs, ne = ctx->G.ne;
    int rc;
    if (!mooring) {
        if ((rc = upload_obs_layout(ctx, obs->xy, nobs))) return rc;
    }
    CK(cudaMemcpyAsync(ctx->d_obs_y, value, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->st));
    // 1-2: innovations, S d, phi
    {
        Phase sub_("innovations");
        KL(1, launch_innovate(ctx->buf[0], ctx->buf[1], ctx->par, ctx->d_cell, ctx->d_obs_y, nobs, ctx->G,
                           ctx->P.H_eq, ctx->d_d, ctx->st));
        if (!mooring && (rc = factor(ctx, nobs))) return rc;
        KL(1, launch_solve(ctx->d_L, ctx->d_colptr, ctx->d_rowidx, ctx->d_rdiag, ctx->d_plan, n, ctx->d_d, ctx->d_Sd,
                           ctx->d_phi, ne, ctx->st, ctx->d_perm_u, ctx->d_xs, mooring ? ctx->d_Lr : nullptr,
                           mooring ? ctx->d_Lc : nullptr));
    }
    // 3: random vectors
    Phase sub_("weights_and_update");
    const uint32_t sb = 16u * (uint32_t)ctx->P.instance_id;
    KL(1, launch_rand_dots(ctx->P.seed, ctx->cycle, sb + 1, sb + 2, (int)ctx->NR, ne, ctx->d_partial,
                        ctx->dots_blk, ctx->st));
    // 4-5: target weight, beta (two-stage), alpha
    KL(1, launch_sync_alpha(ctx->d_phi, ctx->d_partial, ctx->dots_blk, ne, (double)ctx->NR, 3.0 * ctx->plane,
                         std::log((double)ne), ctx->P.scheme, ctx->d_c, ctx->d_gamma, ctx->d_zeta, ctx->d_alpha, ctx->d_cstar,
                         ctx->d_neglogw, ctx->d_coef, ctx->d_scal, ctx->flag, ctx->st));
    // 6: posterior coarse field, local block roots, fused update with the pull
    KL(1, launch_form_r(ctx->P.seed, ctx->cycle, sb + 1, sb + 2, (int)ctx->NR, ne, ctx->d_coef, ctx->d_scal,
                     ctx->d_alpha, ctx->d_r, ctx->st));
    if (mooring && ctx->nblev > 0) {
        KL(1, launch_block_levels(ctx->d_r, (int)ctx->NR, ne, ctx->d_M49, ctx->d_block0, ctx->d_border, ctx->d_blevel,
                                  ctx->nblev, ctx->C.nRx, ctx->C.nRy, ctx->st));
    } else {
        KL(1, launch_block_seq(ctx->d_r, (int)ctx->NR, ne, ctx->d_M49, ctx->d_block0, nobs, ctx->C.nRx, ctx->C.nRy,
                               ctx->st));
    }
    QhalfArgs A{};
    A.b0 = ctx->buf[0];
    A.b1 = ctx->buf[1];
    A.par = ctx->par;
    A.wtab = ctx->d_wtab;
    A.from_philox = 0;
    A.x = ctx->d_r;
    A.with_pull = 1;
    A.K = ctx->d_K32;
    A.R = ctx->R;
    A.obs_cell = ctx->d_cell;
    A.Sd = ctx->d_Sd;
    A.nobs = nobs;
    A.tile_cnt = ctx->d_tile_cnt;
    A.tile_obs = ctx->d_tile_obs;
    A.tile_cap = ctx->tile_cap;
    A.xi_buf = ctx->d_xi;
    A.soar_buf = ctx->d_soar;
    A.amax = ctx->amax;
    CK(cudaMemsetAsync(ctx->amax, 0, sizeof(float) * ne, ctx->st));
    KL(qhalf_launches(A), launch_qhalf(A, ctx->G, ctx->C, ctx->st));
    ctx->cfl_ready = true;
    // diagnostics
    CK(cudaMemcpyAsync(ctx->h_scal, ctx->d_scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    if (diag) {
        double* dst[] = {diag->phi, diag->c, diag->gamma, diag->zeta, diag->alpha, diag->neglogw};
        double* src[] = {ctx->d_phi, ctx->d_c, ctx->d_gamma, ctx->d_zeta, ctx->d_alpha, ctx->d_neglogw};
        for (int i = 0; i < 6; ++i)
            if (dst[i]) CK(cudaMemcpyAsync(dst[i], src[i], sizeof(double) * ne, cudaMemcpyDeviceToHost, ctx->st));
    }
    rc = read_flags(ctx);
    if (diag) {
        diag->w_target = ctx->h_scal[0];
        diag->beta = ctx->h_scal[1];
        diag->c_bar = ctx->h_scal[2];
    }
    ctx->cycle++;
    return rc;
}

int iewpf_sir_weights(iewpf_ctx_t* ctx, const iewpf_obs_t* obs, double r_scale, int n_sets, int set_size,
                      const int* sets, double* w, int* n_kept)
{
    Phase phase_("sir_weights");
    if (!ctx) return IEWPF_EINVAL;
    if (!obs || obs->n_obs < 1 || obs->n_obs > ctx->nobs_max) return fail(ctx, IEWPF_EINVAL, "bad observation set");
    const bool mooring = ctx->P.obs_kind == IEWPF_OBS_MOORING;
    if (!mooring && !obs->xy) return fail(ctx, IEWPF_EINVAL, "drifter observations need positions");
    if (mooring && obs->n_obs != ctx->nobs_max)
        return fail(ctx, IEWPF_EINVAL, "mooring observations must cover every mooring");
    std::vector<double> derived;
    const double* value = obs_values(ctx->P, *obs, derived);
    if (!value) return fail(ctx, IEWPF_EINVAL, "no observed values (and no usable previous drifter fixes)");
    if (!obs_finite(*obs, value)) return fail(ctx, IEWPF_EINVAL, "non-finite observation value or position");
    const int nobs = obs->n_obs, ne = ctx->G.ne;
    if (!(r_scale > 0) || !std::isfinite(r_scale) || n_sets < 0 || set_size < 1 || set_size > nobs ||
        (n_sets > 0 && (!sets || !n_kept)))
        return fail(ctx, IEWPF_EINVAL, "bad observation subsets");
    for (long long k = 0; k < (long long)n_sets * set_size; ++k)
        if (sets[k] < 0 || sets[k] >= nobs) return fail(ctx, IEWPF_EINVAL, "subset index out of range");
    if (n_sets == 0) return IEWPF_OK;
    CK(cudaSetDevice(ctx->dev));
    int rc;
    if (!mooring && (rc = upload_obs_layout(ctx, obs->xy, nobs))) return rc;
    CK(cudaMemcpyAsync(ctx->d_obs_y, value, sizeof(double) * 2 * nobs, cudaMemcpyHostToDevice, ctx->st));
    KL(1, launch_innovate(ctx->buf[0], ctx->buf[1], ctx->par, ctx->d_cell, ctx->d_obs_y, nobs, ctx->G,
                       ctx->P.H_eq, ctx->d_d, ctx->st));
    const size_t nidx = (size_t)n_sets * set_size, nw = (size_t)n_sets * ne;
    int* d_sets = nullptr;
    int* d_kept = nullptr;
    double* d_w = nullptr;
    if (cudaMalloc((void**)&d_sets, sizeof(int) * nidx) != cudaSuccess ||
        cudaMalloc((void**)&d_kept, sizeof(int) * n_sets) != cudaSuccess ||
        cudaMalloc((void**)&d_w, sizeof(double) * nw) != cudaSuccess) {
        cudaFree(d_sets);
        cudaFree(d_kept);
        cudaFree(d_w);
        cudaGetLastError();
        return fail(ctx, IEWPF_ENOMEM, "subset buffers");
    }
    const double sigma2 = ctx->P.obs_sigma * ctx->P.obs_sigma;
    cudaError_t e = cudaMemcpyAsync(d_sets, sets, sizeof(int) * nidx, cudaMemcpyHostToDevice, ctx->st);
    if (e == cudaSuccess) {
        e = launch_sir_weights(ctx->d_d, ne, nobs, d_sets, n_sets, set_size, 0.5 / (r_scale * sigma2), d_w, d_kept,
                               ctx->st);
        if (e == cudaSuccess) ctx->launches += 1;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(n_kept, d_kept, sizeof(int) * n_sets, cudaMemcpyDeviceToHost, ctx->st);
    if (e == cudaSuccess && w) e = cudaMemcpyAsync(w, d_w, sizeof(double) * nw, cudaMemcpyDeviceToHost, ctx->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
    cudaFree(d_sets);
    cudaFree(d_kept);
    cudaFree(d_w);
    if (e != cudaSuccess) return fail(ctx, IEWPF_ECUDA, cudaGetErrorString(e));
    return read_flags(ctx);
}

int iewpf_rank(iewpf_ctx_t* ctx, int n_pts, const int* cells, const double* y, uint32_t draw, int* ranks)
{
    Phase phase_("rank");
    if (!ctx) return IEWPF_EINVAL;
    if (n_pts < 1 || !cells || !y || !ranks) return fail(ctx, IEWPF_EINVAL, "bad rank points");
    for (int m = 0; m < n_pts; ++m)
        if (cells[2 * m] < 0 || cells[2 * m] >= ctx->G.nx || cells[2 * m + 1] < 0 || cells[2 * m + 1] >= ctx->G.ny ||
            !std::isfinite(y[2 * m]) || !std::isfinite(y[2 * m + 1]))
            return fail(ctx, IEWPF_EINVAL, "rank point outside the grid or non-finite value");
    CK(cudaSetDevice(ctx->dev));
    int* d_cells = nullptr;
    int* d_ranks = nullptr;
    double* d_y = nullptr;
    if (cudaMalloc((void**)&d_cells, sizeof(int) * 2 * n_pts) != cudaSuccess ||
        cudaMalloc((void**)&d_ranks, sizeof(int) * 2 * n_pts) != cudaSuccess ||
        cudaMalloc((void**)&d_y, sizeof(double) * 2 * n_pts) != cudaSuccess) {
        cudaFree(d_cells);
        cudaFree(d_ranks);
        cudaFree(d_y);
        cudaGetLastError();
        return fail(ctx, IEWPF_ENOMEM, "rank buffers");
    }
    const uint32_t stream = 16u * (uint32_t)ctx->P.instance_id + 3u;
    cudaError_t e = cudaMemcpyAsync(d_cells, cells, sizeof(int) * 2 * n_pts, cudaMemcpyHostToDevice, ctx->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_y, y, sizeof(double) * 2 * n_pts, cudaMemcpyHostToDevice, ctx->st);
    if (e == cudaSuccess) {
        e = launch_rank(ctx->buf[0], ctx->buf[1], ctx->par, ctx->G, d_cells, d_y, n_pts, ctx->P.seed, draw, stream,
                        ctx->P.obs_sigma, d_ranks, ctx->st);
        if (e == cudaSuccess) ctx->launches += 1;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ranks, d_ranks, sizeof(int) * 2 * n_pts, cudaMemcpyDeviceToHost, ctx->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
    cudaFree(d_cells);
    cudaFree(d_ranks);
    cudaFree(d_y);
    if (e != cudaSuccess) return fail(ctx, IEWPF_ECUDA, cudaGetErrorString(e));
    return IEWPF_OK;
}

int iewpf_set_drifters(iewpf_ctx_t* ctx, const double* xy, int n)
{
    if (!ctx) return IEWPF_EINVAL;
    if (n < 0 || n > ctx->P.n_drifters_max || (n > 0 && !xy)) return fail(ctx, IEWPF_EINVAL, "bad drifters");
    CK(cudaSetDevice(ctx->dev));
    ctx->nd = n;
    if (n > 0) {
        CK(cudaMemcpyAsync(ctx->d_xy, xy, sizeof(double) * 2 * n * ctx->G.ne, cudaMemcpyHostToDevice, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
    }
    return IEWPF_OK;
}

int iewpf_get_drifters(iewpf_ctx_t* ctx, double* xy)
{
    if (!ctx) return IEWPF_EINVAL;
    if (!xy) return fail(ctx, IEWPF_EINVAL, "null pointer");
    CK(cudaSetDevice(ctx->dev));
    if (ctx->nd > 0) {
        CK(cudaMemcpyAsync(xy, ctx->d_xy, sizeof(double) * 2 * ctx->nd * ctx->G.ne, cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
    }
    return IEWPF_OK;
}

int drifter_forecast(iewpf_ctx_t* ctx, const double* xy0, int n, double hours, double out_every_s, double* traj,
                     int use_surrogate)
{
    Phase phase_("drifter_forecast");
    if (!ctx) return IEWPF_EINVAL;
    if (use_surrogate && !ctx->sur) return fail(ctx, IEWPF_EINVAL, "no surrogate attached (iewpf_set_surrogate)");
    if (!xy0 || !traj || n < 1 || n > ctx->P.n_drifters_max || !(hours >= 0) || !(out_every_s > 0))
        return fail(ctx, IEWPF_EINVAL, "bad drifter forecast arguments");
    const double ratio = out_every_s / ctx->P.dt_model;
    const int every = (int)std::lround(ratio);
    if (every < 1 || std::fabs(ratio - every) > 1e-9)
        return fail(ctx, IEWPF_EINVAL, "out_every_s must be a multiple of dt_model");
    const int n_out = (int)std::floor(hours * 3600.0 / out_every_s + 1e-9) + 1;
    const int ne = ctx->G.ne;
    std::vector<double> rep((size_t)ne * n * 2);
    for (int p = 0; p < ne; ++p) std::memcpy(&rep[(size_t)p * n * 2], xy0, sizeof(double) * 2 * n);
    int rc;
    if ((rc = iewpf_set_drifters(ctx, rep.data(), n))) return rc;
    const size_t per = (size_t)ne * n * 2;
    std::memcpy(traj, rep.data(), sizeof(double) * per);
    if (use_surrogate && every % ctx->sur_k != 0)
        return fail(ctx, IEWPF_EINVAL, "out_every_s must be a multiple of the surrogate's k model steps");
    for (int o = 1; o < n_out; ++o) {
        if (use_surrogate) {
            for (int c = 0; c < every / ctx->sur_k; ++c)
                if ((rc = surrogate_steps(ctx))) return rc;
        } else if ((rc = iewpf_forecast(ctx, every, 1))) {
            return rc;
        }
        if ((rc = iewpf_get_drifters(ctx, traj + per * o))) return rc;
    }
    return IEWPF_OK;
}

int drifter_forecast_errors(iewpf_ctx_t* ctx, const double* xy0, int n, double hours, double out_every_s,
                            const double* truth, double* E, double* RMSE, double* traj, int use_surrogate)
{
    Phase phase_("drifter_forecast");
    if (!ctx) return IEWPF_EINVAL;
    if (!xy0 || !truth || !E || !RMSE || n < 1 || n > ctx->P.n_drifters_max || !(hours >= 0) || !(out_every_s > 0))
        return fail(ctx, IEWPF_EINVAL, "bad drifter forecast arguments");
    const double ratio = out_every_s / ctx->P.dt_model;
    const int every = (int)std::lround(ratio);
    if (every < 1 || std::fabs(ratio - every) > 1e-9)
        return fail(ctx, IEWPF_EINVAL, "out_every_s must be a multiple of dt_model");
    CK(cudaSetDevice(ctx->dev));
    const int n_out = (int)std::floor(hours * 3600.0 / out_every_s + 1e-9) + 1;
    const int ne = ctx->G.ne;
    const size_t per = (size_t)ne * n * 2;
    std::vector<double> rep(per);
    for (int p = 0; p < ne; ++p) std::memcpy(&rep[(size_t)p * n * 2], xy0, sizeof(double) * 2 * n);
    int rc;
    if ((rc = iewpf_set_drifters(ctx, rep.data(), n))) return rc;
    double *d_truth = nullptr, *d_err = nullptr, *d_traj = nullptr;
    auto cleanup = [&]() {
        if (d_truth) cudaFree(d_truth);
        if (d_err) cudaFree(d_err);
        if (d_traj) cudaFree(d_traj);
    };
    if ((rc = dalloc(ctx, &d_truth, (size_t)n_out * n * 2)) || (rc = dalloc(ctx, &d_err, 2 * (size_t)n_out)) ||
        (traj && (rc = dalloc(ctx, &d_traj, per * n_out)))) {
        cleanup();
        return rc;
    }
    auto body = [&]() -> int {
        CK(cudaMemcpyAsync(d_truth, truth, sizeof(double) * n_out * n * 2, cudaMemcpyHostToDevice, ctx->st));
        if (use_surrogate && (!ctx->sur || every % ctx->sur_k != 0))
            return fail(ctx, IEWPF_EINVAL, "surrogate missing or k does not divide the output interval");
        for (int o = 0; o < n_out; ++o) {
            int r;
            if (o > 0 && use_surrogate) {
                for (int c = 0; c < every / ctx->sur_k; ++c)
                    if ((r = surrogate_steps(ctx))) return r;
            } else if (o > 0 && (r = iewpf_forecast(ctx, every, 1))) {
                return r;
            }
            KL(1, launch_drift_errors(ctx->d_xy, d_truth + (size_t)o * n * 2, ne, n, d_err + o, d_err + n_out + o,
                                      ctx->st));
            if (traj)
                CK(cudaMemcpyAsync(d_traj + per * o, ctx->d_xy, sizeof(double) * per, cudaMemcpyDeviceToDevice,
                                   ctx->st));
        }
        CK(cudaMemcpyAsync(E, d_err, sizeof(double) * n_out, cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaMemcpyAsync(RMSE, d_err + n_out, sizeof(double) * n_out, cudaMemcpyDeviceToHost, ctx->st));
        if (traj) CK(cudaMemcpyAsync(traj, d_traj, sizeof(double) * per * n_out, cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        return IEWPF_OK;
    };
    rc = body();
    cleanup();
    return rc;
}

int iewpf_save(const iewpf_ctx_t* cctx, const char* path)
{
    iewpf_ctx* ctx = const_cast<iewpf_ctx*>(cctx);
    if (!ctx) return IEWPF_EINVAL;
    if (!path) return fail(ctx, IEWPF_EINVAL, "null path");
    const size_t nstate = (size_t)ctx->G.ne * 3 * ctx->plane;
    std::vector<float> st(nstate);
    int rc = iewpf_get_state(ctx, st.data(), 0, nullptr);
    if (rc) return rc;
    std::vector<double> xy((size_t)ctx->G.ne * 2 * std::max(ctx->nd, 0));
    if (ctx->nd > 0 && (rc = iewpf_get_drifters(ctx, xy.data()))) return rc;
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(ctx, IEWPF_EINVAL, std::string("cannot open ") + path);
    const uint32_t magic = 0x46505749u;   // "IWPF"
    const int32_t hdr[5] = {ctx->P.nx, ctx->P.ny, ctx->G.ne, ctx->nd, 1};
    bool ok = std::fwrite(&magic, 4, 1, f) == 1 && std::fwrite(hdr, 4, 5, f) == 5 &&
              std::fwrite(&ctx->step, 4, 1, f) == 1 && std::fwrite(&ctx->cycle, 4, 1, f) == 1 &&
              std::fwrite(st.data(), 4, nstate, f) == nstate &&
              (xy.empty() || std::fwrite(xy.data(), 8, xy.size(), f) == xy.size());
    ok = (std::fclose(f) == 0) && ok;
    return ok ? IEWPF_OK : fail(ctx, IEWPF_EINVAL, "write failed");
}

int iewpf_load(iewpf_ctx_t* ctx, const char* path)
{
    if (ctx) ctx->cfl_ready = false;
    if (!ctx) return IEWPF_EINVAL;
    if (!path) return fail(ctx, IEWPF_EINVAL, "null path");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(ctx, IEWPF_EINVAL, std::string("cannot open ") + path);
    uint32_t magic = 0, step = 0, cyc = 0;
    int32_t hdr[5] = {0};
    bool ok = std::fread(&magic, 4, 1, f) == 1 && std::fread(hdr, 4, 5, f) == 5 &&
              std::fread(&step, 4, 1, f) == 1 && std::fread(&cyc, 4, 1, f) == 1;
    if (!ok || magic != 0x46505749u || hdr[0] != ctx->P.nx || hdr[1] != ctx->P.ny || hdr[2] != ctx->G.ne ||
        hdr[3] < 0 || hdr[3] > ctx->P.n_drifters_max) {
        std::fclose(f);
        return fail(ctx, IEWPF_EINVAL, "checkpoint does not match this context");
    }
    const size_t nstate = (size_t)ctx->G.ne * 3 * ctx->plane;
    std::vector<float> st(nstate);
    std::vector<double> xy((size_t)ctx->G.ne * 2 * hdr[3]);
    ok = std::fread(st.data(), 4, nstate, f) == nstate && (xy.empty() || std::fread(xy.data(), 8, xy.size(), f) == xy.size());
    std::fclose(f);
    if (!ok) return fail(ctx, IEWPF_EINVAL, "truncated checkpoint");
    int rc = iewpf_set_state(ctx, st.data(), 0, nullptr);
    if (rc) return rc;
    if ((rc = iewpf_set_drifters(ctx, xy.data(), hdr[3]))) return rc;
    ctx->step = step;
    ctx->cycle = cyc;
    return IEWPF_OK;
}

int iewpf_get_counters(const iewpf_ctx_t* ctx, uint32_t* model_step, uint32_t* cycle)
{
    if (!ctx) return IEWPF_EINVAL;
    if (model_step) *model_step = ctx->step;
    if (cycle) *cycle = ctx->cycle;
    return IEWPF_OK;
}

int iewpf_set_counters(iewpf_ctx_t* ctx, uint32_t model_step, uint32_t cycle)
{
    if (!ctx) return IEWPF_EINVAL;
    ctx->step = model_step;
    ctx->cycle = cycle;
    return IEWPF_OK;
}

int iewpf_last_nsub(const iewpf_ctx_t* cctx, int* n_sub)
{
    iewpf_ctx* ctx = const_cast<iewpf_ctx*>(cctx);
    if (!ctx) return IEWPF_EINVAL;
    if (!n_sub) return fail(ctx, IEWPF_EINVAL, "null pointer");
    CK(cudaSetDevice(ctx->dev));
    CK(cudaMemcpyAsync(n_sub, ctx->nsub, sizeof(int) * ctx->G.ne, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return IEWPF_OK;
}

const char* iewpf_last_error(const iewpf_ctx_t* ctx)
{
    return ctx ? ctx->err.c_str() : kNullMsg;
}

int iewpf_philox_blocks(uint64_t seed, uint32_t p, uint32_t t, uint32_t stream, int64_t n_blocks, uint32_t* out)
{
    if (!out || n_blocks < 0) return IEWPF_EINVAL;
    uint32_t* d = nullptr;
    if (cudaMalloc((void**)&d, sizeof(uint32_t) * 4 * (size_t)std::max<int64_t>(n_blocks, 1)) != cudaSuccess)
        return IEWPF_ENOMEM;
    int rc = IEWPF_OK;
    if (launch_philox_blocks(seed, p, t, stream, n_blocks, d, 0) != cudaSuccess ||
        cudaMemcpy(out, d, sizeof(uint32_t) * 4 * (size_t)n_blocks, cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = IEWPF_ECUDA;
    cudaFree(d);
    return rc;
}

int iewpf_normals(uint64_t seed, uint32_t p, uint32_t t, uint32_t stream, int64_t n, double* out64, float* out32)
{
    if (n < 0 || (!out64 && !out32)) return IEWPF_EINVAL;
    double* d64 = nullptr;
    float* d32 = nullptr;
    const size_t m = (size_t)std::max<int64_t>(n, 1);
    if ((out64 && cudaMalloc((void**)&d64, 8 * m) != cudaSuccess) ||
        (out32 && cudaMalloc((void**)&d32, 4 * m) != cudaSuccess)) {
        if (d64) cudaFree(d64);
        return IEWPF_ENOMEM;
    }
    int rc = IEWPF_OK;
    if (launch_normals(seed, p, t, stream, n, d64, d32, 0) != cudaSuccess ||
        (out64 && cudaMemcpy(out64, d64, 8 * (size_t)n, cudaMemcpyDeviceToHost) != cudaSuccess) ||
        (out32 && cudaMemcpy(out32, d32, 4 * (size_t)n, cudaMemcpyDeviceToHost) != cudaSuccess))
        rc = IEWPF_ECUDA;
    if (d64) cudaFree(d64);
    if (d32) cudaFree(d32);
    return rc;
}

static int weights_host(int scheme, int ne, double N_psi, const double* c, const double* gamma, const double* zeta,
                        double* out2, double* alpha, double* cstar, double* neglogw)
{
    if (ne < 1 || !(N_psi > 0) || !c || !gamma || !zeta || !out2 || !alpha || !cstar) return IEWPF_EINVAL;
    double* d = nullptr;
    int* flag = nullptr;
    const size_t n = (size_t)ne;
    if (cudaMalloc((void**)&d, sizeof(double) * (6 * n + 4)) != cudaSuccess) return IEWPF_ENOMEM;
    if (cudaMalloc((void**)&flag, sizeof(int)) != cudaSuccess) {
        cudaFree(d);
        return IEWPF_ENOMEM;
    }
    double *dc = d, *dg = d + n, *dz = d + 2 * n, *da = d + 3 * n, *ds = d + 4 * n, *dw = d + 5 * n,
           *dsc = d + 6 * n;
    int rc = IEWPF_OK, hf = 0;
    if (cudaMemset(flag, 0, sizeof(int)) != cudaSuccess ||
        cudaMemcpy(dc, c, 8 * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dg, gamma, 8 * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dz, zeta, 8 * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        launch_weights_only(dc, dg, dz, ne, N_psi, scheme, da, ds, dw, dsc, flag, 0) != cudaSuccess ||
        cudaMemcpy(out2, dsc, 16, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(alpha, da, 8 * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(cstar, ds, 8 * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
        (neglogw && cudaMemcpy(neglogw, dw, 8 * n, cudaMemcpyDeviceToHost) != cudaSuccess) ||
        cudaMemcpy(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = IEWPF_ECUDA;
    cudaFree(d);
    cudaFree(flag);
    if (rc == IEWPF_OK && hf) {
        if (hf & FLAG_NONFINITE) rc = IEWPF_ENONFINITE;
        else if (hf & FLAG_BETA) rc = IEWPF_EBETA;
        else if (hf & FLAG_DOMAIN) rc = IEWPF_EDOMAIN;
    }
    return rc;
}

int iewpf_weights(int ne, double N_psi, const double* c, const double* gamma, const double* zeta, double* out2,
                  double* alpha, double* cstar, double* neglogw)
{
    return weights_host(IEWPF_TWO_STAGE, ne, N_psi, c, gamma, zeta, out2, alpha, cstar, neglogw);
}

int iewpf_drifter_obs(const iewpf_params_t* params, int n, const double* xy, const double* xy_prev, double dt,
                      double* value)
{
    if (!params || !(params->dx > 0) || !(params->dy > 0) || params->nx < 1 || params->ny < 1) return IEWPF_EINVAL;
    return drifter_obs_values(params->nx * params->dx, params->ny * params->dy, params->H_eq, n, xy, xy_prev, dt, value);
}

int iewpf_alpha_gamma(int ne, double N_psi, const double* gamma, const double* cstar, double* alpha)
{
    Phase phase_("alpha_gamma");
    if (ne < 1 || !(N_psi > 0) || !std::isfinite(N_psi) || !gamma || !cstar || !alpha) return IEWPF_EINVAL;
    for (int i = 0; i < ne; ++i)
        if (!(gamma[i] > 0) || !std::isfinite(gamma[i]) || !(cstar[i] >= 0) || !std::isfinite(cstar[i]))
            return IEWPF_EINVAL;
    double* d = nullptr;
    int* flag = nullptr;
    const size_t n = (size_t)ne;
    if (cudaMalloc((void**)&d, sizeof(double) * 3 * n) != cudaSuccess) return IEWPF_ENOMEM;
    if (cudaMalloc((void**)&flag, sizeof(int)) != cudaSuccess) {
        cudaFree(d);
        return IEWPF_ENOMEM;
    }
    int rc = IEWPF_OK, hf = 0;
    if (cudaMemset(flag, 0, sizeof(int)) != cudaSuccess ||
        cudaMemcpy(d, gamma, 8 * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d + n, cstar, 8 * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        launch_alpha_gamma(ne, N_psi, d, d + n, d + 2 * n, flag, 0) != cudaSuccess ||
        cudaMemcpy(alpha, d + 2 * n, 8 * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = IEWPF_ECUDA;
    cudaFree(d);
    cudaFree(flag);
    if (rc == IEWPF_OK && hf) rc = IEWPF_EDOMAIN;
    return rc;
}

int iewpf_weights_one_stage(int ne, double N_psi, const double* c, const double* gamma, double* out2,
                            double* alpha, double* cstar, double* neglogw)
{
    // zeta is not read by the one-stage step; gamma stands in for the pointer
    return weights_host(IEWPF_ONE_STAGE, ne, N_psi, c, gamma, gamma, out2, alpha, cstar, neglogw);
}

int iewpf_pull_stencil(const iewpf_ctx_t* ctx, double* K)
{
    if (!ctx || !K) return IEWPF_EINVAL;
    std::memcpy(K, ctx->K64.data(), sizeof(double) * ctx->K64.size());
    return IEWPF_OK;
}

int iewpf_local_block(const iewpf_ctx_t* ctx, double* M)
{
    if (!ctx || !M) return IEWPF_EINVAL;
    std::memcpy(M, ctx->M49.data(), sizeof(double) * ctx->M49.size());
    return IEWPF_OK;
}

int iewpf_block_levels(const int* block0, int nobs, int nRx, int nRy, int* level)
{
    if (nobs < 0 || nRx < 1 || nRy < 1 || (nobs > 0 && (!block0 || !level))) return IEWPF_EINVAL;
    for (int l = 0; l < nobs; ++l)
        if (block0[2 * l] < 0 || block0[2 * l] >= nRx || block0[2 * l + 1] < 0 || block0[2 * l + 1] >= nRy)
            return IEWPF_EINVAL;
    std::vector<int> order, off;
    block_levels(block0, nobs, nRx, nRy, order, off);
    for (size_t v = 0; v + 1 < off.size(); ++v)
        for (int i = off[v]; i < off[v + 1]; ++i) level[order[i]] = (int)v;
    return IEWPF_OK;
}

int iewpf_add_qhalf(iewpf_ctx_t* ctx, const float* x)
{
    if (ctx) ctx->cfl_ready = false;
    if (!ctx) return IEWPF_EINVAL;
    if (!x) return fail(ctx, IEWPF_EINVAL, "null pointer");
    CK(cudaSetDevice(ctx->dev));
    CK(cudaMemcpyAsync(ctx->d_r, x, sizeof(float) * ctx->NR * ctx->G.ne, cudaMemcpyHostToDevice, ctx->st));
    QhalfArgs A{};
    A.b0 = ctx->buf[0];
    A.b1 = ctx->buf[1];
    A.par = ctx->par;
    A.wtab = ctx->d_wtab;
    A.from_philox = 0;
    A.x = ctx->d_r;
    A.xi_buf = ctx->d_xi;
    A.soar_buf = ctx->d_soar;
    KL(qhalf_launches(A), launch_qhalf(A, ctx->G, ctx->C, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return IEWPF_OK;
}

int iewpf_stream(const iewpf_ctx_t* ctx, void** stream)
{
    if (!ctx || !stream) return IEWPF_EINVAL;
    *stream = (void*)ctx->st;
    return IEWPF_OK;
}

int iewpf_substeps(iewpf_ctx_t* ctx, int n, double dt)
{
    if (ctx) ctx->cfl_ready = false;
    if (!ctx) return IEWPF_EINVAL;
    if (n < 0 || !(dt > 0)) return fail(ctx, IEWPF_EINVAL, "bad substep arguments");
    CK(cudaSetDevice(ctx->dev));
    int rc;
    if (!ctx->tuned && (rc = tune_stepper(ctx))) return rc;
    std::vector<int> ones(ctx->G.ne, n);
    std::vector<float> dts(ctx->G.ne, (float)dt);
    CK(cudaMemcpyAsync(ctx->nsub, ones.data(), sizeof(int) * ones.size(), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->dtp, dts.data(), sizeof(float) * dts.size(), cudaMemcpyHostToDevice, ctx->st));
    for (int s = 0; s < n; ++s) KL(1, launch_step(ctx, s));
    KL(1, launch_par_update(ctx->par, ctx->nsub, ctx->G.ne, ctx->work, ctx->st));
    // the host vectors must outlive the copies
    CK(cudaStreamSynchronize(ctx->st));
    return IEWPF_OK;
}

int iewpf_work(iewpf_ctx_t* ctx, int64_t* particle_substeps)
{
    if (!ctx || !particle_substeps) return IEWPF_EINVAL;
    CK(cudaSetDevice(ctx->dev));
    unsigned long long w = 0;
    CK(cudaMemcpyAsync(&w, ctx->work, sizeof(w), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    *particle_substeps = (int64_t)w;
    return IEWPF_OK;
}

int iewpf_set_stepper(iewpf_ctx_t* ctx, int kind, int nc, int rows, int warps)
{
    if (!ctx) return IEWPF_EINVAL;
    if ((kind != 1 && kind != 2) || (nc != 2 && nc != 3 && nc != 4) || rows < 1 || warps < 1 || warps > 8)
        return fail(ctx, IEWPF_EINVAL, "bad stepper shape");
    ctx->stepper = kind;
    ctx->shape = MarchShape{nc, rows, warps, kind == 2};
    ctx->tuned = true;
    return IEWPF_OK;
}

int iewpf_tune(iewpf_ctx_t* ctx, int* shape)
{
    if (!ctx) return IEWPF_EINVAL;
    CK(cudaSetDevice(ctx->dev));
    int rc = tune_stepper(ctx);
    if (rc) return rc;
    if (shape) {
        shape[0] = ctx->stepper;
        shape[1] = ctx->shape.nc;
        shape[2] = ctx->shape.TH;
        shape[3] = ctx->shape.warps;
    }
    return IEWPF_OK;
}

int iewpf_get_stepper(const iewpf_ctx_t* ctx, int* shape)
{
    if (!ctx || !shape) return IEWPF_EINVAL;
    shape[0] = ctx->stepper;
    shape[1] = ctx->shape.nc;
    shape[2] = ctx->shape.TH;
    shape[3] = ctx->shape.warps;
    return IEWPF_OK;
}

int iewpf_launch_count(const iewpf_ctx_t* ctx, int64_t* count)
{
    if (!ctx || !count) return IEWPF_EINVAL;
    *count = ctx->launches;
    return IEWPF_OK;
}

int iewpf_factor_info(iewpf_ctx_t* ctx, int* n_y, int64_t* nnz_L)
{
    if (!ctx) return IEWPF_EINVAL;
    CK(cudaSetDevice(ctx->dev));
    int nnz = 0;
    if (ctx->n_fact > 0) {
        CK(cudaMemcpyAsync(&nnz, ctx->d_colptr + ctx->n_fact, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
    }
    if (n_y) *n_y = ctx->n_fact;
    if (nnz_L) *nnz_L = nnz;
    return IEWPF_OK;
}

int iewpf_sizes(const iewpf_ctx_t* ctx, int* nRx, int* nRy, int* stencil_R)
{
    if (!ctx) return IEWPF_EINVAL;
    if (nRx) *nRx = ctx->C.nRx;
    if (nRy) *nRy = ctx->C.nRy;
    if (stencil_R) *stencil_R = ctx->R;
    return IEWPF_OK;
}

// ---------------------------------------------------------------------------
// batched problems
// ---------------------------------------------------------------------------
struct iewpf_batch {
    std::vector<iewpf_ctx*> inst;
    BatchImpl* impl = nullptr;
    cudaStream_t st = nullptr, st2 = nullptr;
    int dev = 0;
    std::string err;
};

static int bfail(iewpf_batch* b, int code, const std::string& msg)
{
    if (b) b->err = msg;
    return code;
}

#define BCK(call)                                                                                    \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return bfail(b, IEWPF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));        \
    } while (0)

int iewpf_batch_destroy(iewpf_batch_t* b)
{
    if (!b) return IEWPF_OK;
    cudaSetDevice(b->dev);
    if (b->st) cudaStreamSynchronize(b->st);
    batch_delete(b->impl);
    for (iewpf_ctx* c : b->inst) iewpf_destroy(c);
    if (b->st) cudaStreamDestroy(b->st);
    if (b->st2) cudaStreamDestroy(b->st2);
    delete b;
    return IEWPF_OK;
}

int iewpf_batch_create(const iewpf_params_t* params, const double* const* mooring_xy, int n, iewpf_batch_t** out)
{
    Phase phase_("batch_create");
    if (!params || !out || n < 1) return IEWPF_EINVAL;
    *out = nullptr;
    iewpf_batch* b = new (std::nothrow) iewpf_batch();
    if (!b) return IEWPF_ENOMEM;
    cudaGetDevice(&b->dev);
    std::vector<BInst> desc;
    for (int i = 0; i < n; ++i) {
        iewpf_ctx* ctx = nullptr;
        if (params[i].n_obs_max < 1) {
            iewpf_batch_destroy(b);
            return IEWPF_EINVAL;
        }
        int rc = iewpf_create(&params[i], mooring_xy ? mooring_xy[i] : nullptr, &ctx);
        if (rc) {
            iewpf_batch_destroy(b);
            return rc;
        }
        b->inst.push_back(ctx);
        BInst I{};
        I.step = march::StepArgs{ctx->buf[0], ctx->buf[1], ctx->par, ctx->nsub, ctx->dtp, ctx->G, 64, 0, 0};
        I.b0 = ctx->buf[0];
        I.b1 = ctx->buf[1];
        I.par = ctx->par;
        I.nsub = ctx->nsub;
        I.dtp = ctx->dtp;
        I.amax = ctx->amax;
        I.G = ctx->G;
        I.C = ctx->C;
        I.courant = ctx->P.courant;
        I.dt_model = ctx->P.dt_model;
        I.wtab = ctx->d_wtab;
        I.seed = ctx->P.seed;
        I.stream_base = 16u * (uint32_t)ctx->P.instance_id;
        I.work = ctx->work;
        I.flag = ctx->flag;
        I.nobs = ctx->nobs_max;
        I.moving_obs = ctx->P.obs_kind == IEWPF_OBS_DRIFTER;
        I.dx = ctx->P.dx;
        I.dy = ctx->P.dy;
        I.H = ctx->P.H_eq;
        I.sigma2 = ctx->P.obs_sigma * ctx->P.obs_sigma;
        I.dense = ctx->P.dense_S;
        I.scheme = ctx->P.scheme;
        I.R = ctx->R;
        I.cell = ctx->d_cell;
        I.block0 = ctx->d_block0;
        I.tile_cnt = ctx->d_tile_cnt;
        I.tile_obs = ctx->d_tile_obs;
        I.tile_cap = ctx->tile_cap;
        I.K64 = ctx->d_K64;
        I.K32 = ctx->d_K32;
        I.M49 = ctx->d_M49;
        I.L = ctx->d_L;
        I.rdiag = ctx->d_rdiag;
        I.plan = ctx->d_plan;
        I.colptr = ctx->d_colptr;
        I.rowidx = ctx->d_rowidx;
        I.perm = ctx->d_perm_u;
        I.xs = ctx->d_xs;
        I.Lr = ctx->d_Lr;
        I.Lc = ctx->d_Lc;
        I.d = ctx->d_d;
        I.Sd = ctx->d_Sd;
        I.phi = ctx->d_phi;
        I.partial = ctx->d_partial;
        I.nblk = ctx->dots_blk;
        I.c = ctx->d_c;
        I.gamma = ctx->d_gamma;
        I.zeta = ctx->d_zeta;
        I.alpha = ctx->d_alpha;
        I.cstar = ctx->d_cstar;
        I.neglogw = ctx->d_neglogw;
        I.coef = ctx->d_coef;
        I.scal = ctx->d_scal;
        I.r = ctx->d_r;
        I.xi = ctx->d_xi;
        I.soar = ctx->d_soar;
        I.NR = ctx->NR;
        I.N_psi = 3.0 * ctx->plane;
        I.logNe = std::log((double)ctx->G.ne);
        desc.push_back(I);
    }
    b->impl = batch_new();
    if (!b->impl) {
        iewpf_batch_destroy(b);
        return IEWPF_ENOMEM;
    }
    if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->st2, cudaStreamNonBlocking) != cudaSuccess ||
        batch_init(*b->impl, desc) != cudaSuccess) {
        cudaGetLastError();
        iewpf_batch_destroy(b);
        return IEWPF_ENOMEM;
    }
    *out = b;
    return IEWPF_OK;
}

int iewpf_batch_instance(iewpf_batch_t* b, int i, iewpf_ctx_t** ctx)
{
    if (!b || !ctx || i < 0 || i >= (int)b->inst.size()) return IEWPF_EINVAL;
    *ctx = b->inst[i];
    return IEWPF_OK;
}

int iewpf_batch_tune(iewpf_batch_t* b, int* shape)
{
    if (!b) return IEWPF_EINVAL;
    BCK(cudaSetDevice(b->dev));
    BCK(batch_tune(*b->impl, b->st));
    if (shape) batch_shape(*b->impl, shape);
    return IEWPF_OK;
}

int iewpf_batch_cycle(iewpf_batch_t* b, int n_model_steps, const iewpf_obs_t* obs, double* diag)
{
    Phase phase_("batch_cycle");
    if (!b) return IEWPF_EINVAL;
    if (n_model_steps < 1 || !obs) return bfail(b, IEWPF_EINVAL, "bad cycle arguments");
    const int n = (int)b->inst.size();
    for (int i = 0; i < n; ++i) {
        const iewpf_ctx* c = b->inst[i];
        const bool mooring = c->P.obs_kind == IEWPF_OBS_MOORING;
        if (obs[i].n_obs != c->nobs_max || (!mooring && !obs[i].xy))
            return bfail(b, IEWPF_EINVAL, "problem " + std::to_string(i) + ": observations must fill n_obs_max");
    }
    std::vector<std::vector<double>> derived(n);
    std::vector<const double*> values(n);
    for (int i = 0; i < n; ++i) {
        values[i] = obs_values(b->inst[i]->P, obs[i], derived[i]);
        if (!values[i]) return bfail(b, IEWPF_EINVAL, "problem " + std::to_string(i) + ": no observed values");
        if (!obs_finite(obs[i], values[i]))
            return bfail(b, IEWPF_EINVAL, "problem " + std::to_string(i) + ": non-finite observation");
    }
    BCK(cudaSetDevice(b->dev));
    if (!batch_tuned(*b->impl)) BCK(batch_tune(*b->impl, b->st));
    // inputs into the pinned staging the graph reads
    for (int i = 0; i < n; ++i) {
        double* dst = batch_obs_staging(*b->impl, i);
        const int m = obs[i].n_obs;
        if (obs[i].xy) std::memcpy(dst, obs[i].xy, sizeof(double) * 2 * m);
        else std::memset(dst, 0, sizeof(double) * 2 * m);
        std::memcpy(dst + 2 * m, values[i], sizeof(double) * 2 * m);
        uint32_t* ctr = batch_counter_staging(*b->impl);
        ctr[2 * i] = b->inst[i]->step;
        ctr[2 * i + 1] = b->inst[i]->cycle;
    }
    for (int i = 0; i < n; ++i) b->inst[i]->cfl_ready = false;
    BCK(batch_cycle(*b->impl, n_model_steps, b->st, b->st2));
    BCK(cudaStreamSynchronize(b->st));
    const double* dg = batch_diag(*b->impl);
    int rc = IEWPF_OK;
    for (int i = 0; i < n; ++i) {
        iewpf_ctx* c = b->inst[i];
        c->step += (uint32_t)n_model_steps;
        c->cycle += 1;
        if (diag) std::memcpy(diag + 3 * i, dg + 3 * i, 3 * sizeof(double));
        const int f = (int)dg[3 * i + 2];
        if (f && rc == IEWPF_OK) {
            rc = check_flags(c, f);
            b->err = "problem " + std::to_string(i) + ": " + c->err;
        }
    }
    return rc;
}

int iewpf_batch_forecast(iewpf_batch_t* b, int n_model_steps, int add_model_error)
{
    Phase phase_("batch_forecast");
    if (!b) return IEWPF_EINVAL;
    if (n_model_steps < 1) return bfail(b, IEWPF_EINVAL, "n_model_steps < 1");
    const int n = (int)b->inst.size();
    BCK(cudaSetDevice(b->dev));
    if (!batch_tuned(*b->impl)) BCK(batch_tune(*b->impl, b->st));
    uint32_t* ctr = batch_counter_staging(*b->impl);
    for (int i = 0; i < n; ++i) {
        ctr[2 * i] = b->inst[i]->step;
        ctr[2 * i + 1] = b->inst[i]->cycle;
        b->inst[i]->cfl_ready = false;
    }
    BCK(batch_forecast(*b->impl, n_model_steps, add_model_error != 0, b->st, b->st2));
    BCK(cudaStreamSynchronize(b->st));
    const double* dg = batch_diag(*b->impl);
    int rc = IEWPF_OK;
    for (int i = 0; i < n; ++i) {
        iewpf_ctx* c = b->inst[i];
        c->step += (uint32_t)n_model_steps;
        const int f = (int)dg[3 * i + 2];
        if (f && rc == IEWPF_OK) {
            rc = check_flags(c, f);
            b->err = "problem " + std::to_string(i) + ": " + c->err;
        }
    }
    return rc;
}

int iewpf_batch_stream(const iewpf_batch_t* b, void** stream)
{
    if (!b || !stream) return IEWPF_EINVAL;
    *stream = (void*)b->st;
    return IEWPF_OK;
}

int iewpf_batch_work(iewpf_batch_t* b, int64_t* particle_substeps, int64_t* launches)
{
    if (!b) return IEWPF_EINVAL;
    BCK(cudaSetDevice(b->dev));
    unsigned long long w = 0;
    BCK(batch_work(*b->impl, &w));
    if (particle_substeps) *particle_substeps = (int64_t)w;
    if (launches) *launches = batch_launches(*b->impl);
    return IEWPF_OK;
}

const char* iewpf_batch_last_error(const iewpf_batch_t* b)
{
    return b ? b->err.c_str() : kNullMsg;
}

// ---------------------------------------------------------------------------
// learned surrogate
// ---------------------------------------------------------------------------
static int sfail(iewpf_surrogate* s, int code, const std::string& msg)
{
    if (s) s->err = msg;
    return code;
}

#define SCK(call)                                                                                    \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return sfail(s, IEWPF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));        \
    } while (0)

int iewpf_surrogate_set_path(iewpf_surrogate_t* s, int path)
{
    if (!s || path < 0 || path > 1) return IEWPF_EINVAL;
    s->net.path = path;
    return IEWPF_OK;
}

int iewpf_surrogate_get_path(const iewpf_surrogate_t* s, int* uses_tcgen05)
{
    if (!s || !uses_tcgen05) return IEWPF_EINVAL;
    *uses_tcgen05 = (s->net.uses_tc() ? 1 : 0) | (s->net.uses_tc_train() ? 2 : 0);
    return IEWPF_OK;
}

int iewpf_surrogate_destroy(iewpf_surrogate_t* s)
{
    if (!s) return IEWPF_OK;
    cudaSetDevice(s->dev);
    if (s->st) cudaStreamSynchronize(s->st);
    if (s->S0) cudaFree(s->S0);
    if (s->S1) cudaFree(s->S1);
    if (s->stats) cudaFree(s->stats);
    s->net.release();
    if (s->st) cudaStreamDestroy(s->st);
    delete s;
    return IEWPF_OK;
}

int iewpf_surrogate_create(int nx, int ny, int width, int depth, uint64_t seed, iewpf_surrogate_t** out)
{
    if (!out) return IEWPF_EINVAL;
    *out = nullptr;
    iewpf_surrogate* s = new (std::nothrow) iewpf_surrogate();
    if (!s) return IEWPF_ENOMEM;
    cudaGetDevice(&s->dev);
    int rc = s->net.init(nx, ny, width, depth);
    if (rc || cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess) {
        iewpf_surrogate_destroy(s);
        return rc ? rc : IEWPF_ECUDA;
    }
    // He-normal initial weights (fan-in 9 cin), zero biases; the output layer
    // starts small so the initial prediction is close to "no change"
    std::mt19937_64 gen(seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    std::vector<float> p(s->net.n_params, 0.0f);
    for (int l = 0; l < s->net.depth; ++l) {
        const int cin = s->net.layer_cin(l), cout = s->net.layer_cout(l);
        const int real_in = l == 0 ? 3 : cin, real_out = l == s->net.depth - 1 ? 3 : cout;
        const double sd = std::sqrt(2.0 / (9.0 * real_in)) * (l == s->net.depth - 1 ? 0.1 : 1.0);
        for (int tap = 0; tap < 9; ++tap)
            for (int co = 0; co < cout; ++co)
                for (int ci = 0; ci < cin; ++ci)
                    if (co < real_out && ci < real_in)
                        p[s->net.w_off[l] + ((size_t)tap * cout + co) * cin + ci] = (float)(sd * nd(gen));
    }
    if (cudaMemcpyAsync(s->net.master, p.data(), p.size() * 4, cudaMemcpyHostToDevice, s->st) != cudaSuccess ||
        s->net.cast(s->st) != cudaSuccess || cudaStreamSynchronize(s->st) != cudaSuccess) {
        iewpf_surrogate_destroy(s);
        return IEWPF_ECUDA;
    }
    *out = s;
    return IEWPF_OK;
}

int iewpf_surrogate_param_count(const iewpf_surrogate_t* s, int64_t* n)
{
    if (!s || !n) return IEWPF_EINVAL;
    *n = (int64_t)s->net.n_params;
    return IEWPF_OK;
}

int iewpf_surrogate_set_params(iewpf_surrogate_t* s, const float* params)
{
    if (!s || !params) return IEWPF_EINVAL;
    SCK(cudaSetDevice(s->dev));
    SCK(cudaMemcpyAsync(s->net.master, params, s->net.n_params * 4, cudaMemcpyHostToDevice, s->st));
    SCK(s->net.cast(s->st));
    SCK(cudaStreamSynchronize(s->st));
    return IEWPF_OK;
}

int iewpf_surrogate_get_params(const iewpf_surrogate_t* cs, float* params)
{
    iewpf_surrogate* s = const_cast<iewpf_surrogate*>(cs);
    if (!s || !params) return IEWPF_EINVAL;
    SCK(cudaSetDevice(s->dev));
    SCK(cudaMemcpyAsync(params, s->net.master, s->net.n_params * 4, cudaMemcpyDeviceToHost, s->st));
    SCK(cudaStreamSynchronize(s->st));
    return IEWPF_OK;
}

int iewpf_surrogate_set_scales(iewpf_surrogate_t* s, const double* in_scale, const double* out_scale)
{
    if (!s || !in_scale || !out_scale) return IEWPF_EINVAL;
    for (int c = 0; c < 3; ++c) {
        if (!(in_scale[c] > 0) || !(out_scale[c] > 0)) return sfail(s, IEWPF_EINVAL, "scales must be positive");
        s->net.in_scale[c] = (float)in_scale[c];
        s->net.out_scale[c] = (float)out_scale[c];
    }
    return IEWPF_OK;
}

int iewpf_surrogate_get_scales(const iewpf_surrogate_t* s, double* in_scale, double* out_scale)
{
    if (!s || !in_scale || !out_scale) return IEWPF_EINVAL;
    for (int c = 0; c < 3; ++c) {
        in_scale[c] = s->net.in_scale[c];
        out_scale[c] = s->net.out_scale[c];
    }
    return IEWPF_OK;
}

int iewpf_surrogate_inject_timeout(iewpf_surrogate_t* s, int n_evals)
{
    if (!s || n_evals < 0) return IEWPF_EINVAL;
    s->net.inject_timeouts = n_evals;
    return IEWPF_OK;
}

int iewpf_surrogate_apply(iewpf_surrogate_t* s, const float* U, int n, float* Unext)
{
    Phase phase_("surrogate_apply");
    if (!s || !U || !Unext || n < 1) return IEWPF_EINVAL;
    SCK(cudaSetDevice(s->dev));
    const size_t per = 3ull * s->net.nx * s->net.ny;
    float* d = nullptr;
    if (cudaMalloc((void**)&d, per * n * 4) != cudaSuccess) return sfail(s, IEWPF_ENOMEM, "input");
    int rc = IEWPF_OK;
    cudaError_t e = cudaMemcpyAsync(d, U, per * n * 4, cudaMemcpyHostToDevice, s->st);
    for (int p0 = 0; p0 < n && e == cudaSuccess && !rc; p0 += s->chunk) {
        const int nb = std::min(s->chunk, n - p0);
        if (!(rc = s->net.infer(d + per * p0, nb, s->st))) e = s->net.apply(d + per * p0, nb, s->st);
    }
    if (e == cudaSuccess && !rc) e = cudaMemcpyAsync(Unext, d, per * n * 4, cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    cudaFree(d);
    if (rc) return sfail(s, rc, "network");
    if (e != cudaSuccess) return sfail(s, IEWPF_ECUDA, cudaGetErrorString(e));
    return sur_flag(s, s->st);
}

int iewpf_surrogate_apply_device(iewpf_surrogate_t* s, const float* U, int n, float* Unext, void* stream)
{
    Phase phase_("surrogate_apply");
    if (!s || !U || !Unext || n < 1) return IEWPF_EINVAL;
    SCK(cudaSetDevice(s->dev));
    const size_t per = 3ull * s->net.nx * s->net.ny;
    cudaStream_t user = (cudaStream_t)stream;
    cudaEvent_t ev;
    SCK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    int rc = IEWPF_OK;
    cudaError_t e = cudaSuccess;
    if (user && (e = cudaEventRecord(ev, user)) == cudaSuccess) e = cudaStreamWaitEvent(s->st, ev, 0);
    if (e == cudaSuccess && Unext != U) e = cudaMemcpyAsync(Unext, U, per * n * 4, cudaMemcpyDeviceToDevice, s->st);
    for (int p0 = 0; p0 < n && e == cudaSuccess && !rc; p0 += s->chunk) {
        const int nb = std::min(s->chunk, n - p0);
        if (!(rc = s->net.infer(Unext + per * p0, nb, s->st))) e = s->net.apply(Unext + per * p0, nb, s->st);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev, s->st);
    if (e == cudaSuccess) e = user ? cudaStreamWaitEvent(user, ev, 0) : cudaEventSynchronize(ev);
    cudaEventDestroy(ev);
    if (rc) return sfail(s, rc, "network");
    if (e != cudaSuccess) return sfail(s, IEWPF_ECUDA, cudaGetErrorString(e));
    return user ? IEWPF_OK : sur_flag(s, s->st);
}

int iewpf_surrogate_stream(const iewpf_surrogate_t* s, void** stream)
{
    if (!s || !stream) return IEWPF_EINVAL;
    *stream = (void*)s->st;
    return IEWPF_OK;
}

int iewpf_surrogate_loss_grad(iewpf_surrogate_t* s, const float* X, const float* Y, int n, double* loss, float* grad)
{
    if (!s || !X || !Y || n < 1) return IEWPF_EINVAL;
    SCK(cudaSetDevice(s->dev));
    const size_t per = 3ull * s->net.nx * s->net.ny;
    float *dx = nullptr, *dy = nullptr;
    if (cudaMalloc((void**)&dx, per * n * 4) != cudaSuccess || cudaMalloc((void**)&dy, per * n * 4) != cudaSuccess) {
        if (dx) cudaFree(dx);
        return sfail(s, IEWPF_ENOMEM, "pairs");
    }
    int rc = s->net.ensure_batch(n);
    cudaError_t e = cudaSuccess;
    if (!rc) {
        if ((e = cudaMemcpyAsync(dx, X, per * n * 4, cudaMemcpyHostToDevice, s->st)) == cudaSuccess &&
            (e = cudaMemcpyAsync(dy, Y, per * n * 4, cudaMemcpyHostToDevice, s->st)) == cudaSuccess &&
            (e = s->net.pack_input(dx, n, s->st)) == cudaSuccess && (e = s->net.pack_target(dx, dy, n, s->st)) == cudaSuccess &&
            (e = s->net.forward(n, s->st)) == cudaSuccess && (e = s->net.backward(n, s->st)) == cudaSuccess) {
            if (loss) e = cudaMemcpyAsync(loss, s->net.dloss, 8, cudaMemcpyDeviceToHost, s->st);
            if (e == cudaSuccess && grad) e = cudaMemcpyAsync(grad, s->net.grad, s->net.n_params * 4, cudaMemcpyDeviceToHost, s->st);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    }
    cudaFree(dx);
    cudaFree(dy);
    if (rc) return sfail(s, rc, "activations");
    if (e != cudaSuccess) return sfail(s, IEWPF_ECUDA, cudaGetErrorString(e));
    return sur_flag(s, s->st);
}

int iewpf_surrogate_train(iewpf_surrogate_t* s, iewpf_ctx_t* ctx, int n_pairs, int k_steps, int epochs, int batch,
                          double lr, double* epoch_loss)
{
    Phase phase_("surrogate_train");
    if (!s || !ctx || n_pairs < 1 || k_steps < 1 || epochs < 0 || batch < 1 || !(lr > 0)) return IEWPF_EINVAL;
    if (ctx->P.nx != s->net.nx || ctx->P.ny != s->net.ny) return sfail(s, IEWPF_EINVAL, "grid mismatch");
    SCK(cudaSetDevice(s->dev));
    const int ne = ctx->G.ne;
    const size_t per = 3ull * s->net.nx * s->net.ny;
    const int nbat = n_pairs / batch;       // batches per epoch (a last partial batch is skipped)
    const long long total = (long long)epochs * nbat;
    float *X = nullptr, *Y = nullptr, *d_bc = nullptr;
    int* d_order = nullptr;                 // the epoch's order of the pairs; a batch reads its slice
    int* d_ctr = nullptr;                   // batch cursor, optimizer step of this call
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    auto cleanup = [&]() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        for (cudaEvent_t ev : {ev0, ev1})
            if (ev) cudaEventDestroy(ev);
        gexec = nullptr;
        graph = nullptr;
        ev0 = ev1 = nullptr;
        for (void* p : {(void*)X, (void*)Y, (void*)d_order, (void*)d_ctr, (void*)d_bc})
            if (p) cudaFree(p);
        X = Y = d_bc = nullptr;
        d_order = d_ctr = nullptr;
    };
    // from here on a failed CUDA call frees the buffers, graph and events
#undef SCK
#define SCK(call)                                                                                    \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) {                                                                     \
            cleanup();                                                                               \
            return sfail(s, IEWPF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));        \
        }                                                                                            \
    } while (0)
    if (cudaMalloc((void**)&X, per * n_pairs * 4) != cudaSuccess || cudaMalloc((void**)&Y, per * n_pairs * 4) != cudaSuccess ||
        cudaMalloc((void**)&d_order, sizeof(int) * n_pairs) != cudaSuccess ||
        cudaMalloc((void**)&d_ctr, sizeof(int) * 2) != cudaSuccess ||
        cudaMalloc((void**)&d_bc, sizeof(float) * 2 * std::max<long long>(total, 1)) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return sfail(s, IEWPF_ENOMEM, "training pairs");
    }
    int rc = IEWPF_OK;
    // pairs (psi, M^k psi) of the plain scheme without model error (the
    // surrogate stands for the deterministic model; model error is added
    // after it); between pairs the ensemble advances k steps with model error
    float* snap = nullptr;
    if (cudaMalloc((void**)&snap, per * ne * 4) != cudaSuccess) {
        cleanup();
        return sfail(s, IEWPF_ENOMEM, "snapshot");
    }
    // every copy on ctx's stream, behind the forecasts that produce it
    for (int got = 0; got < n_pairs && !rc;) {
        const int take = std::min(ne, n_pairs - got);
        if ((rc = iewpf_get_state(ctx, snap, 1, nullptr))) break;
        if (cudaMemcpyAsync(X + per * got, snap, per * take * 4, cudaMemcpyDeviceToDevice, ctx->st) != cudaSuccess) {
            rc = IEWPF_ECUDA;
            break;
        }
        if ((rc = iewpf_forecast(ctx, k_steps, 0))) break;
        if ((rc = iewpf_get_state(ctx, snap, 1, nullptr))) break;
        if (cudaMemcpyAsync(Y + per * got, snap, per * take * 4, cudaMemcpyDeviceToDevice, ctx->st) != cudaSuccess) {
            rc = IEWPF_ECUDA;
            break;
        }
        if ((rc = iewpf_forecast(ctx, k_steps, 1))) break;
        got += take;
    }
    if (!rc && cudaStreamSynchronize(ctx->st) != cudaSuccess) rc = IEWPF_ECUDA;
    cudaFree(snap);
    if (rc) {
        cleanup();
        return sfail(s, rc, std::string("generating pairs: ") + ctx->err);
    }
    // normalisation from the data (up to 64 pairs spread over the set): input
    // and output change of unit spread per field, one scale for both momentum
    // components (the problem is isotropic in the horizontal)
    {
        const int ns = std::min(n_pairs, 64);
        const size_t plane = (size_t)s->net.nx * s->net.ny;
        std::vector<float> hx(per), hy(per);
        double sx[3] = {0, 0, 0}, sxx[3] = {0, 0, 0}, sd[3] = {0, 0, 0}, sdd[3] = {0, 0, 0};
        for (int q = 0; q < ns; ++q) {
            const size_t pi = (size_t)q * n_pairs / ns;
            cudaMemcpy(hx.data(), X + per * pi, per * 4, cudaMemcpyDeviceToHost);
            cudaMemcpy(hy.data(), Y + per * pi, per * 4, cudaMemcpyDeviceToHost);
            for (int c = 0; c < 3; ++c)
                for (size_t i = 0; i < plane; ++i) {
                    const double x = hx[c * plane + i], d = hy[c * plane + i] - x;
                    sx[c] += x;
                    sxx[c] += x * x;
                    sd[c] += d;
                    sdd[c] += d * d;
                }
        }
        const double cnt = (double)ns * plane;
        auto spread = [&](const double* a, const double* aa, int c0, int c1) {
            double m = 0, v = 0;
            for (int c = c0; c <= c1; ++c) m += a[c];
            m /= cnt * (c1 - c0 + 1);
            for (int c = c0; c <= c1; ++c) v += aa[c];
            v = v / (cnt * (c1 - c0 + 1)) - m * m;
            return std::sqrt(std::max(v, 1e-30));
        };
        const double x_eta = spread(sx, sxx, 0, 0), x_mom = spread(sx, sxx, 1, 2);
        const double d_eta = spread(sd, sdd, 0, 0), d_mom = spread(sd, sdd, 1, 2);
        s->net.in_scale[0] = (float)(1.0 / x_eta);
        s->net.in_scale[1] = s->net.in_scale[2] = (float)(1.0 / x_mom);
        s->net.out_scale[0] = (float)d_eta;
        s->net.out_scale[1] = s->net.out_scale[2] = (float)d_mom;
    }
    if ((rc = s->net.ensure_batch(batch))) {
        cleanup();
        return sfail(s, rc, "activations");
    }
    std::mt19937_64 gen(12345);
    std::vector<int> order(n_pairs);
    for (int i = 0; i < n_pairs; ++i) order[i] = i;
    // Adam's bias corrections of this call's steps (host arithmetic, as adam_step)
    {
        std::vector<float> bc(2 * std::max<long long>(total, 1), 1.0f);
        for (long long k = 0; k < total; ++k) {
            const float t = (float)(s->net.t_adam + 1 + k);
            bc[2 * k] = 1.0f - std::pow(Surrogate::kAdamB1, t);
            bc[2 * k + 1] = 1.0f - std::pow(Surrogate::kAdamB2, t);
        }
        SCK(cudaMemcpyAsync(d_bc, bc.data(), sizeof(float) * bc.size(), cudaMemcpyHostToDevice, s->st));
        SCK(cudaMemsetAsync(d_ctr, 0, sizeof(int) * 2, s->st));
        SCK(cudaStreamSynchronize(s->st));
    }
    // one optimizer step captured as a CUDA graph and replayed per batch: the
    // step reads its batch through the cursor and its bias corrections
    // through the step counter, both in device memory
    if (total > 0) {
        SCK(cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal));
        const cudaError_t ce = s->net.train_step(X, Y, d_order, d_ctr, d_bc, batch, (float)lr, s->st);
        const cudaError_t ee = cudaStreamEndCapture(s->st, &graph);
        SCK(ce);
        SCK(ee);
        SCK(cudaGraphInstantiate(&gexec, graph, 0));
    }
    SCK(cudaEventCreate(&ev0));
    SCK(cudaEventCreate(&ev1));
    SCK(cudaEventRecord(ev0, s->st));
    // the batches of an epoch are queued without a host synchronisation; the
    // batch losses add up on the device and are read once per epoch
    for (int ep = 0; ep < epochs; ++ep) {
        for (int i = n_pairs - 1; i > 0; --i) std::swap(order[i], order[gen() % (uint64_t)(i + 1)]);
        SCK(cudaMemcpyAsync(d_order, order.data(), sizeof(int) * n_pairs, cudaMemcpyHostToDevice, s->st));
        SCK(cudaMemsetAsync(d_ctr, 0, sizeof(int), s->st));
        SCK(cudaMemsetAsync(s->net.eloss, 0, sizeof(double), s->st));
        for (int k = 0; k < nbat; ++k) SCK(cudaGraphLaunch(gexec, s->st));
        double acc = 0.0;
        SCK(cudaMemcpyAsync(&acc, s->net.eloss, 8, cudaMemcpyDeviceToHost, s->st));
        SCK(cudaStreamSynchronize(s->st));
        if (epoch_loss) epoch_loss[ep] = nbat ? acc / nbat : 0.0;
    }
    s->net.t_adam += (int)total;
    SCK(cudaEventRecord(ev1, s->st));
    SCK(cudaEventSynchronize(ev1));
    float ms = 0.0f;
    SCK(cudaEventElapsedTime(&ms, ev0, ev1));
    s->train_s = ms * 1e-3;
    cleanup();
    return sur_flag(s, s->st);
}
#undef SCK
#define SCK(call)                                                                                    \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return sfail(s, IEWPF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));        \
    } while (0)

int iewpf_surrogate_train_time(const iewpf_surrogate_t* s, double* seconds)
{
    if (!s || !seconds) return IEWPF_EINVAL;
    *seconds = s->train_s;
    return IEWPF_OK;
}

int iewpf_set_surrogate(iewpf_ctx_t* ctx, iewpf_surrogate_t* s, int k_steps)
{
    if (!ctx) return IEWPF_EINVAL;
    if (s && (k_steps < 1 || s->net.nx != ctx->P.nx || s->net.ny != ctx->P.ny))
        return fail(ctx, IEWPF_EINVAL, "surrogate grid or k mismatch");
    ctx->sur = s;
    ctx->sur_k = s ? k_steps : 0;
    return IEWPF_OK;
}

int iewpf_surrogate_stats(const iewpf_ctx_t* ctx, int64_t* calls, int64_t* fallbacks)
{
    if (!ctx) return IEWPF_EINVAL;
    if (calls) *calls = ctx->sur_calls;
    if (fallbacks) *fallbacks = ctx->sur_fallbacks;
    return IEWPF_OK;
}

const char* iewpf_surrogate_last_error(const iewpf_surrogate_t* s)
{
    return s ? s->err.c_str() : kNullMsg;
}

}  // extern "C"
