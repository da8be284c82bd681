// mlp.h -- the contact-detection schedule network: 16 -> 64 -> 64 -> 2 with ReLU, BF16
// operands on the tensor cores (mma.sync m16n8k16), FP32 accumulation, FP32 master
// weights trained with Adam on the GPU.
//
// Parameters, flat FP32: W1[64][16], b1[64], W2[64][64], b2[64], W3[2][64], b3[2].
// Outputs: (log2 of the steps until the largest accumulated displacement in a bin
// exceeds the margin, the same for half the margin).  Loss: mean over rows and outputs of
// w * (y_hat - y)^2 with w = 4 where the prediction overshoots (an overshoot costs an
// audit fallback) and 1 otherwise.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

namespace dem {

constexpr int MLP_IN = 16, MLP_H = 64, MLP_OUT = 2;
constexpr int MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_OUT * MLP_H + MLP_OUT;
constexpr float MLP_OVERSHOOT_WEIGHT = 4.0f;

class Mlp {
public:
    Mlp() = default;
    ~Mlp();
    // Xavier-uniform weights from a 64-bit seed (splitmix64 stream), zero biases.
    cudaError_t init(uint64_t seed, cudaStream_t st);
    cudaError_t set_params(const float *host_params, cudaStream_t st);
    cudaError_t get_params(float *host_params, cudaStream_t st);
    // out[rows][2] = net(X[rows][16]); X and out on the device (FP32).
    cudaError_t forward(const float *X, int rows, float *out, cudaStream_t st);
    // loss and gradient of the loss for device X[rows][16], Y[rows][2] (gradient on host).
    cudaError_t loss_grad(const float *X, const float *Y, int rows, float *loss, float *grad_host, cudaStream_t st);
    // Adam epochs over host data X[n][16], Y[n][2] with seeded shuffling; mean loss of the
    // last epoch in *loss.
    cudaError_t train(const std::vector<float> &X, const std::vector<float> &Y, int epochs, float lr, uint64_t seed,
                      float *loss, cudaStream_t st);
    bool ready() const { return ready_; }

private:
    cudaError_t reserve(int rows);
    cudaError_t step_batch(const float *X, const float *Y, int rows, float *loss_out, cudaStream_t st, bool update,
                           float lr, int t);
    bool ready_ = false;
    float *w_ = nullptr;        // FP32 master parameters
    uint16_t *wb_ = nullptr;    // BF16 copy
    float *g_ = nullptr, *m_ = nullptr, *v_ = nullptr;
    int cap_ = 0;               // rows of the scratch below
    uint16_t *xb_ = nullptr, *h1b_ = nullptr, *h2b_ = nullptr, *dob_ = nullptr, *dh2b_ = nullptr, *dh1b_ = nullptr;
    float *h1_ = nullptr, *h2_ = nullptr, *out_ = nullptr, *dout_ = nullptr, *dh2_ = nullptr, *dh1_ = nullptr;
    float *lossp_ = nullptr;
    float *xg_ = nullptr, *yg_ = nullptr;   // gathered minibatch
    int *idx_ = nullptr;
};

}  // namespace dem
