// Host side of the learned surrogate (surrogate.cu): parameters, buffers and
// the forward / backward / Adam passes of the periodic 3x3 convolutional
// network on one nx x ny grid.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"

namespace iewpf {

#ifdef __CUDACC__
// SiLU(z) = z sigmoid(z) with sigmoid(z) = (1 + tanh(z / 2)) / 2 from the
// hardware tanh approximation: h + h tanh(h), h = z / 2 (one MUFU operation)
__device__ __forceinline__ float tanh_approx(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float silu_act(float z)
{
    const float h = 0.5f * z;
    return fmaf(h, tanh_approx(h), h);
}
// d SiLU / dz = s (1 + z (1 - s)), s = sigmoid(z)
__device__ __forceinline__ float silu_grad(float z)
{
    const float s = fmaf(0.5f, tanh_approx(0.5f * z), 0.5f);
    return s * fmaf(z, 1.0f - s, 1.0f);
}
#endif

struct Surrogate {
    int nx = 0, ny = 0, width = 64, depth = 6;
    size_t n_params = 0;
    std::vector<size_t> w_off, b_off;       // offsets of each layer's weights / bias in the flat parameters
    float* master = nullptr;                // fp32 parameters
    float* grad = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    int t_adam = 0;
    std::vector<__nv_bfloat16*> wf, wd;     // bf16 weights: forward [tap][co][ci], backward-data [tap][ci][co]
    // activations for a batch
    int cap_batch = 0;
    __nv_bfloat16* x_in = nullptr;          // [b][ny][nx][16]
    std::vector<__nv_bfloat16*> z, a;       // per hidden layer [b][ny][nx][64]
    float* out = nullptr;                   // [b][ny][nx][3]
    float* target = nullptr;                // [b][ny][nx][3]
    __nv_bfloat16 *dz_a = nullptr, *dz_b = nullptr, *dz_out = nullptr;
    float* wpartial = nullptr;
    float* bpartial = nullptr;
    double* lpartial = nullptr;
    double* dloss = nullptr;
    double* eloss = nullptr;                // running sum of batch losses (training)
    // training on the tcgen05 kernels (conv_tr.cu, uses_tc_train()): x_in,
    // a[l], dz_out, dz_a and dz_b carry a one-pixel periodic halo,
    // [b][ny + 2][nx + 2][C]; z stays [b][ny][nx][64]
    int batch_pad = 0;                      // layout of the batch buffers: 1 = halo-padded
    CUtensorMap tm_in;                      // x_in as layer 0's input
    std::vector<CUtensorMap> tm_fwd;        // a[l] as layer l + 1's input
    std::vector<CUtensorMap> tm_wx;         // a[l] as the X halo patch of layer l + 1's weight gradient
    CUtensorMap tm_dout_f, tm_dout_w;       // dz_out: input of the data pass, dZ of the weight gradient
    CUtensorMap tm_dz_f[2], tm_dz_w[2];     // dz_a, dz_b: the same
    // inference on the tcgen05 kernels: activations with a one-pixel periodic
    // halo, [b][ny + 2][nx + 2][C], and their TMA tensor maps
    int cap_infer = 0;
    __nv_bfloat16* xp = nullptr;            // network input, 16 channels
    __nv_bfloat16* ap[2] = {nullptr, nullptr};
    float* out_i = nullptr;                 // [b][ny][nx][3]
    CUtensorMap map_x, map_a[2];
    float* y_out = nullptr;                 // output of the last infer(): out or out_i
    int path = 0;                           // inference convolutions: 0 tcgen05 where the grid allows, 1 mma.sync
    int* dflag = nullptr;                   // FLAG_TIMEOUT of the tensor-core kernel
    int inject_timeouts = 0;                // network calls left whose tensor-core kernels time out on purpose
    float in_scale[3] = {1.0f, 1.0f, 1.0f};     // network input = state * in_scale
    float out_scale[3] = {1.0f, 1.0f, 1.0f};    // state change = output * out_scale
    std::vector<void*> owned;

    ~Surrogate();
    void release();
    int init(int nx, int ny, int width, int depth);
    int ensure_batch(int nb);
    int wgrad_groups(int nb) const;
    int wgrad9_groups(int nb) const;
    int layer_cin(int l) const;
    int layer_cout(int l) const;
    size_t layer_w(int l) const;
    cudaError_t cast(cudaStream_t st);
    // fields idx[0..nb) of U (or X, Y), fields 0..nb without idx
    // (idx[*cursor + b] with a cursor in device memory)
    cudaError_t pack_input(const float* U, int nb, cudaStream_t st, const int* idx = nullptr,
                           const int* cursor = nullptr);
    cudaError_t pack_target(const float* X, const float* Y, int nb, cudaStream_t st, const int* idx = nullptr,
                            const int* cursor = nullptr);
    // training forward (keeps z for the backward pass; tcgen05 when
    // uses_tc_train(), else mma.sync); output in `out`
    cudaError_t forward(int nb, cudaStream_t st);
    bool uses_tc_train() const;
    // inference: U [nb][3][ny][nx] -> y_out (tcgen05 when uses_tc()); IEWPF code
    int infer(const float* U, int nb, cudaStream_t st);
    int ensure_infer(int nb);
    bool uses_tc() const;
    // loss into dloss (and added to eloss when add_eloss), gradients into grad
    cudaError_t backward(int nb, cudaStream_t st, bool add_eloss = false);
    cudaError_t adam_step(float lr, cudaStream_t st);
    // one optimizer step on the pairs order[ctr[0] .. ctr[0] + batch) of X,
    // Y: pack, forward, backward (loss added to eloss), Adam with the bias
    // corrections bc[2 ctr[1]], bc[2 ctr[1] + 1], weight casts; then ctr[0]
    // += batch and ctr[1] += 1.  Every argument a step reads or advances is in
    // device memory, so the step can be captured once and replayed.
    cudaError_t train_step(const float* X, const float* Y, const int* order, int* ctr, const float* bc, int batch,
                           float lr, cudaStream_t st);
    static constexpr float kAdamB1 = 0.9f, kAdamB2 = 0.999f, kAdamEps = 1e-8f;
    cudaError_t apply(float* U, int nb, cudaStream_t st);
};

// tcgen05 inference convolution (conv_tc.cu) on halo-padded activations:
// layer_kind 0 = 16 -> 64 channels and 1 = 64 -> 64 (bias + SiLU into the
// padded `a`, halo images included), 2 = 64 -> 16 (bias only, first 3 channels
// into f as FP32 [b][ny][nx][3]).  in_map: 16 channels as a 5-D map
// (8 ch, nx+2, ny+2, 2, b) without swizzle, box (8, 130, 4, 2, 1); 64
// channels as a 4-D map (64 ch, nx+2, ny+2, b) with the 128-byte swizzle, box
// (64, 130, 4, 1).  Needs nx % 128 == 0 and ny % 2 == 0.  probe_polls > 0
// injects a timeout: every CTA first waits at most that many polls on a
// barrier nothing completes, then aborts without issuing a copy or product
// and records FLAG_TIMEOUT (tests of the timeout path); 0 runs normally.
bool conv_tc_supported(int nx, int ny);
cudaError_t launch_conv_tc(int layer_kind, const CUtensorMap& in_map, const __nv_bfloat16* W, const float* bias,
                           int nb, int ny, int nx, __nv_bfloat16* a, float* f, int* flag, int probe_polls,
                           cudaStream_t st);

// tcgen05 training convolutions (conv_tr.cu) on halo-padded activations,
// tiles of 16 rows x 8 pixels (with the weight gradients' tiles of 4 rows x
// 64 pixels: needs nx % 64 == 0, ny % 16 == 0).  kind 0 =
// 16 -> 64 and 1 = 64 -> 64 forward (z = conv + bias into z [b][ny][nx][64],
// SiLU(z) into the padded a with its halo images); 2 = 64 -> 16 forward
// (bias added, first 3 channels into f [b][ny][nx][3] FP32); 3 = 16 -> 64 and
// 4 = 64 -> 64 data pass (conv with the flipped transposed weights times
// SiLU'(zprev), zprev [b][ny][nx][64], into the padded a).  in_map: 16
// channels as a 5-D map (8 ch, nx+2, ny+2, 2, b), box (8, 10, 18, 2, 1), no
// swizzle; 64 channels as a 4-D map (64 ch, nx+2, ny+2, b), box (64, 10, 18,
// 1), 128-byte swizzle.
bool conv_tr_supported(int nx, int ny);
cudaError_t launch_conv_tr(int kind, const CUtensorMap& in_map, const __nv_bfloat16* W, const float* bias, int nb,
                           int ny, int nx, __nv_bfloat16* z, __nv_bfloat16* a, float* f, const __nv_bfloat16* zprev,
                           int* flag, cudaStream_t st);
// weight and bias gradients of a 64 -> cout layer (cout 64 or 16) on
// tcgen05: partial [groups][wgrad_tc_partial(cout)], each group's sums over
// its pixel tiles of dW[tap][co][ci] (9 x cout x 64) followed by db[co]
// (cout); adding the groups in order gives the layer's weights and bias in
// the flat parameter layout.  x_map: X (64 ch) as a 4-D map, box (64,
// 66, 6, 1), 128-byte swizzle; d_map: dZ, cout 64 as a 4-D map with box
// (64, 64, 4, 1) and the 128-byte swizzle, cout 16 as a 5-D map with box
// (8, 64, 4, 2, 1) without swizzle.  groups and tiles_per_group from
// wgrad_tc_split.
void wgrad_tc_split(int nb, int ny, int nx, int* groups, int* tiles_per_group);
int wgrad_tc_partial(int cout);
// kernel attributes and device properties the launchers query, set and
// cached outside any stream capture
cudaError_t conv_tr_prepare();
cudaError_t launch_wgrad_tc(int cout, const CUtensorMap& x_map, const CUtensorMap& d_map, int nb, int ny, int nx,
                            int groups, int tiles_per_group, float* partial, int* flag, cudaStream_t st);

// drifters advected over T seconds with the mean of the cell velocities of the
// states before (S0) and after (S1), both [ne][3][ny][nx]
cudaError_t launch_sur_drift(const float* S0, const float* S1, int ne, int nd, double* xy, const Grid& G, double dx,
                             double dy, double T, cudaStream_t st);

// per particle (max |eta|, max velocity component) of S [ne][3][ny][nx] into
// out[ne][2]; +inf for eta when a value is not finite or a depth not positive
cudaError_t launch_sur_stats(const float* S, int ne, const Grid& G, float* out, cudaStream_t st);

}  // namespace iewpf
