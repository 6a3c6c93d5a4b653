// Host interface of the batched IEWPF (batch.cu): the device descriptor of
// one problem and the operations on a batch of problems.
#pragma once
#include <vector>

#include "kernels.h"

namespace iewpf {

// Everything a batched kernel needs of one problem (device pointers into the
// problem's own context).
struct BInst {
    march::StepArgs step;
    float* b0;
    float* b1;
    int* par;
    int* nsub;
    float* dtp;
    float* amax;
    Grid G;
    Coarse C;
    double courant, dt_model;
    const float* wtab;
    uint64_t seed;
    uint32_t stream_base;
    uint32_t* step_ctr;      // model-step draw counter (device)
    uint32_t* cycle;         // cycle draw counter (device)
    unsigned long long* work;
    int* flag;
    // analysis
    int nobs;
    int moving_obs;          // drifters: cells, lists and HQH^T redone every cycle
    double dx, dy, H, sigma2;
    int dense, R;
    int scheme;              // 0 two-stage, 1 one-stage IEWPF
    const double* obs_xy;
    const double* obs_y;
    int* cell;
    int* block0;
    int* tile_cnt;
    int* tile_obs;
    int tile_cap;
    const double* K64;
    const float* K32;
    const float* M49;
    double* L;
    int* colptr;
    int* rowidx;
    double* rdiag;              // level-scheduled solves (ana::solve_plan_cta)
    int* plan;
    const int* perm;            // elimination order of the factor (null: observation order)
    double* xs;                 // [ne][2 nobs] solve scratch when perm is set
    const double* Lr;           // packed factor values of a fixed layout (launch_pack_factor; null: dense reads)
    const double* Lc;
    double* d;
    double* Sd;
    double* phi;
    double* partial;
    int nblk;
    double* c;
    double* gamma;
    double* zeta;
    double* alpha;
    double* cstar;
    double* neglogw;
    double* coef;
    double* scal;
    float* r;
    float* xi;               // coarse normals [ne][N_R] (model error)
    float* soar;             // SOAR coarse field [ne][N_R]
    long long NR;
    double N_psi, logNe;
};

struct BatchImpl;
BatchImpl* batch_new();
void batch_delete(BatchImpl* b);
cudaError_t batch_init(BatchImpl& b, const std::vector<BInst>& insts);
cudaError_t batch_set_step_shape(BatchImpl& b, int nc, int th, int warps, int paired);
cudaError_t batch_tune(BatchImpl& b, cudaStream_t st);
cudaError_t batch_cycle(BatchImpl& b, int n_steps, cudaStream_t st, cudaStream_t st2);
cudaError_t batch_forecast(BatchImpl& b, int n_steps, bool err, cudaStream_t st, cudaStream_t st2);
double* batch_obs_staging(BatchImpl& b, int i);
uint32_t* batch_counter_staging(BatchImpl& b);
const double* batch_diag(const BatchImpl& b);
cudaError_t batch_work(BatchImpl& b, unsigned long long* out);
long long batch_launches(const BatchImpl& b);
void batch_shape(const BatchImpl& b, int* shape);
bool batch_tuned(const BatchImpl& b);

}  // namespace iewpf
