// Host-side launchers of the IEWPF device kernels (internal interface
// between the C ABI in api.cu and the kernel translation units).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace iewpf {

// ---- stepper.cu -----------------------------------------------------------
// have_amax: amax already holds the CFL rates of the current state (left by
// the model-error or analysis update); only n_sub is derived then
cudaError_t launch_cfl(const float* b0, const float* b1, const int* par, float* amax, int* nsub, float* dtp,
                       int* maxsub, const Grid& G, double courant, double dt_model, int fixed,
                       cudaStream_t st, bool have_amax = false,
                       int* flag = nullptr);
cudaError_t launch_par_update(int* par, const int* nsub, int ne, unsigned long long* work, cudaStream_t st);
// the scheme-step loop of a captured model step: reset the index, then after
// every step advance it and keep looping while it is below the largest n_sub
// (and below kMaxSubSingle); the model-step counter of the model error
constexpr int kMaxSubSingle = 100000;
// fixed observation layouts from this size on are factored in a nested-dissection order
constexpr int kNdMinObs = 256;
cudaError_t launch_step_reset(int* s_dev, cudaStream_t st);
cudaError_t launch_step_ctl(int* s_dev, const int* maxsub, cudaGraphConditionalHandle h, unsigned int* iters,
                            cudaStream_t st);
cudaError_t launch_counter_inc(uint32_t* t_dev, cudaStream_t st);
// s_dev (may be null): the scheme-step index read from device memory instead of s
cudaError_t launch_drift(const float* b0, const float* b1, const int* par, const int* nsub, const float* dtp,
                         double* xy, int nd, int s, const Grid& G, double dx, double dy, cudaStream_t st,
                         const int* s_dev = nullptr);
cudaError_t launch_drift_errors(const double* xy, const double* truth, int ne, int nd, double* E, double* RMSE,
                                cudaStream_t st);
cudaError_t launch_nonfinite(const float* b0, const float* b1, const int* par, const Grid& G, int* flag,
                             cudaStream_t st);

// ---- ensemble_stats.cu ----------------------------------------------------
// standard particle filter weights of every particle against n_sets subsets
// of the innovations d [ne][nobs][2]: w [n_sets][ne], kept [n_sets]
cudaError_t launch_sir_weights(const double* d, int ne, int nobs, const int* sets, int n_sets, int set_size,
                               double inv2R, double* w, int* kept, cudaStream_t st);
// ranks [npts][2] of the observed (hu, hv) y [npts][2] at cells [npts][2]
// among the members perturbed by sigma times normals of Philox stream
// `stream`, draw t
cudaError_t launch_rank(const float* b0, const float* b1, const int* par, const Grid& G, const int* cells,
                        const double* y, int npts, uint64_t seed, uint32_t t, uint32_t stream, double sigma,
                        int* ranks, cudaStream_t st);

// ---- alpha_gamma.cu -------------------------------------------------------
// alpha of the incomplete-gamma form of the implicit equation per particle
cudaError_t launch_alpha_gamma(int ne, double N_psi, const double* gamma, const double* cstar, double* alpha,
                               int* flag, cudaStream_t st);

// ---- march.cu -------------------------------------------------------------
namespace march {
// Arguments of one scheme step of one problem.
struct StepArgs {
    float* buf0;
    float* buf1;
    const int* par;
    const int* nsub;
    const float* dtp;
    Grid G;
    int TH, n_strips, n_chunks;
    const int* s_dev = nullptr;   // scheme-step index in device memory (graph loops), else the kernel argument
};
}  // namespace march

// tile shape of the register-marching scheme step: NC columns per lane, TH
// rows per chunk, warps per CTA, and whether the two Runge-Kutta stages run
// paired in packed f32x2 registers (march_warp_paired) or one after the other
// in scalar registers (march_warp)
struct MarchShape {
    int nc, TH, warps;
    int paired = 0;
};
cudaError_t launch_rk2_march(float* b0, float* b1, const int* par, const int* nsub, const float* dtp, int s,
                             const Grid& G, const MarchShape& shape, cudaStream_t st,
                             const int* s_dev = nullptr);

// ---- qhalf.cu -------------------------------------------------------------
// psi += Q^{1/2} x (+ the optimal-proposal pull) for every particle.
struct QhalfArgs {
    float* b0;
    float* b1;
    const int* par;
    const float* wtab;        // SOAR weights by fine offset [tab][tab]
    // source of the coarse field: Philox (model error) or a device array
    int from_philox;
    uint64_t seed;
    uint32_t t;
    const uint32_t* t_dev;    // if set, the draw counter is read from device memory
    uint32_t stream;
    const float* x;           // [ne][N_R]
    // optimal-proposal pull (may be disabled)
    int with_pull;
    const float* K;           // [2][3][2R+1][2R+1]
    int R;
    const int* obs_cell;      // [nobs][2]
    const double* Sd;         // [ne][2 nobs]
    int nobs;
    const int* tile_cnt;      // [ntiles]
    const int* tile_obs;      // [ntiles][tile_cap]
    int tile_cap;
    // optional scratch [ne][N_R] (both or neither): when given, the coarse
    // stages run once per coarse point in their own launches (normals, SOAR)
    // and the fine tiles only interpolate; results are the same bit for bit
    float* xi_buf;
    float* soar_buf;
    // optional [ne], zeroed by the caller: the split path's fine kernel also
    // leaves the CFL rate max of the updated state here (as cfl_kernel would)
    float* amax;
};
// psi += Q^{1/2} x in three stages (normals, SOAR, fine tiles; the normals
// only when x comes from Philox), which need the coarse scratch xi_buf and
// soar_buf (cudaErrorInvalidValue without); qhalf_launches gives the count
cudaError_t launch_qhalf(const QhalfArgs& A, const Grid& G, const Coarse& C, cudaStream_t st);
int qhalf_launches(const QhalfArgs& A);

// ---- analysis.cu ----------------------------------------------------------
cudaError_t launch_obs_setup(const double* xy, int nobs, const Grid& G, const Coarse& C, double dx, double dy,
                             int R, int* obs_cell, int* obs_block0, int* tile_cnt, int* tile_obs, int tile_cap,
                             int* flag, cudaStream_t st);
cudaError_t launch_innovate(const float* b0, const float* b1, const int* par, const int* obs_cell,
                            const double* y, int nobs, const Grid& G, double H, double* d, cudaStream_t st);
cudaError_t launch_hqht(const double* K64, int R, const int* obs_cell, int nobs, const Grid& G, int dense,
                        double sigma2, double* M, cudaStream_t st);
// ints of the level schedule of the triangular sweeps of an n x n factor
__host__ __device__ inline size_t solve_plan_ints(int n)
{
    return 12 * (size_t)n + 5 + (size_t)n * (n - 1) / 2;
}
// FP64 Cholesky of M (n x n) in place, the CSC of the factor below the
// diagonal, its reciprocal diagonal and the level schedule of the two
// triangular sweeps (plan: ana::solve_plan_ints(n) ints)
cudaError_t launch_cholesky(double* M, int n, int* colptr, int* rowidx, int* flag, double* rdiag, int* plan,
                            cudaStream_t st);
// largest vector a particle's solve keeps in shared memory (a CTA of one warp
// per particle); larger systems sweep in global memory
constexpr size_t kSolveSmemBytes = 48 * 1024;
// perm, scratch: see ana::solve_levels_warp (both null: observation order);
// Lr, Lc: the packed values of launch_pack_factor (both null: the sweeps
// read the dense factor)
cudaError_t launch_solve(const double* L, const int* colptr, const int* rowidx, const double* rdiag, const int* plan,
                         int n, const double* d, double* Sd, double* phi, int ne, cudaStream_t st,
                         const int* perm = nullptr, double* scratch = nullptr, const double* Lr = nullptr,
                         const double* Lc = nullptr);
// after launch_cholesky: the factor's values below the diagonal in the order
// of the plan's rows (Lr) and of the CSC (Lc), n (n - 1) / 2 doubles each at
// most
cudaError_t launch_pack_factor(const double* L, int n, const int* colptr, const int* rowidx, const int* plan,
                               double* Lr, double* Lc, cudaStream_t st);
cudaError_t launch_rand_dots(uint64_t seed, uint32_t t, uint32_t s_xi, uint32_t s_nu, int NR, int ne,
                             double* partial, int nblk, cudaStream_t st);
int rand_dots_blocks(int NR);
cudaError_t launch_sync_alpha(const double* phi, const double* partial, int nblk, int ne, double NR,
                              double N_psi, double logNe, int scheme /*0 two-stage, 1 one-stage*/,
                              double* c, double* gamma, double* zeta,
                              double* alpha, double* cstar, double* neglogw, double* coef /*[ne][2]*/,
                              double* scal /*[4]: w_target, beta, mean c*/, int* flag, cudaStream_t st);
cudaError_t launch_weights_only(const double* c, const double* gamma, const double* zeta, int ne, double N_psi,
                                int scheme, double* alpha, double* cstar, double* neglogw, double* scal, int* flag,
                                cudaStream_t st);
cudaError_t launch_form_r(uint64_t seed, uint32_t t, uint32_t s_xi, uint32_t s_nu, int NR, int ne,
                          const double* coef, const double* scal, const double* alpha, float* r,
                          cudaStream_t st);
cudaError_t launch_block_seq(float* r, int NR, int ne, const float* M49, const int* obs_block0, int nobs, int nRx,
                             int nRy, cudaStream_t st);
// the same products level by level (block_levels: order and level_off in
// device memory, nlev levels; the blocks of a level pairwise share no coarse
// point), one CTA per particle whose warps share each level's blocks, the
// same arithmetic as block_seq, so the result is block_seq's bit for bit
cudaError_t launch_block_levels(float* r, int NR, int ne, const float* M49, const int* obs_block0, const int* order,
                                const int* level_off, int nlev, int nRx, int nRy, cudaStream_t st);
// host: level of each block (0 when it shares no coarse point with an earlier
// block, else one more than the highest level among the earlier blocks it
// overlaps; blocks are 7 x 7 coarse points around block0 on the periodic
// nRx x nRy grid).  order = the blocks sorted by level (observation order
// within a level); level_off[v] .. level_off[v + 1] = the range of level v.
void block_levels(const int* block0, int nobs, int nRx, int nRy, std::vector<int>& order,
                  std::vector<int>& level_off);
// host: a nested-dissection elimination order of the observations (cells
// [nobs][2] on the periodic nx x ny grid; two observations are coupled when
// their cells are at most `reach` cells apart in both directions, minimum
// image): recursive bisection of the coupling graph by breadth-first level
// sets, each separator ordered after the two parts it separates.  order[k] =
// the observation eliminated k-th.  Returns the number of coupled pairs.
long long nd_order(const int* cells, int nobs, int nx, int ny, int reach, std::vector<int>& order);
cudaError_t launch_philox_blocks(uint64_t seed, uint32_t p, uint32_t t, uint32_t stream, long long n,
                                 uint32_t* out, cudaStream_t st);
cudaError_t launch_normals(uint64_t seed, uint32_t p, uint32_t t, uint32_t stream, long long n, double* o64,
                           float* o32, cudaStream_t st);

// error flags set by device code
enum : int {
    FLAG_NOTPD = 1,
    FLAG_BETA = 2,
    FLAG_DOMAIN = 4,
    FLAG_NONFINITE = 8,
    FLAG_TILE_OVERFLOW = 16,
    FLAG_TIMEOUT = 32,          // a bounded wait of a tensor-core kernel ran out
};

}  // namespace iewpf
