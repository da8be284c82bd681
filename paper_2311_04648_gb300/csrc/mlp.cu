// mlp.cu -- tensor-core forward, backward and Adam update of the schedule network.
//
// Every matrix product runs through one kernel, k_gemm_bf16: a warp computes a 16x8 tile
// of C = A B with mma.sync.m16n8k16 (BF16 operands, FP32 accumulation), operands read
// row-major or transposed with zero fill outside the matrix, so the same kernel serves
// X W^T (forward), dY W (input gradient) and dY^T H (weight gradient, reduced over the
// batch in a fixed order: deterministic).  The shapes are tiny (K = 16 or 64, N <= 64,
// M = rows): a 128-wide tcgen05 tile with its TMEM and descriptor set-up would sit idle.
#include <algorithm>
#include <cmath>
#include <cstring>

#include <cuda_bf16.h>

#include "mlp.h"

namespace dem {

namespace {

constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + MLP_H * MLP_IN;
constexpr int OFF_W2 = OFF_B1 + MLP_H;
constexpr int OFF_B2 = OFF_W2 + MLP_H * MLP_H;
constexpr int OFF_W3 = OFF_B2 + MLP_H;
constexpr int OFF_B3 = OFF_W3 + MLP_OUT * MLP_H;

__device__ __forceinline__ uint16_t f2bf(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ uint32_t pack2(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

__device__ __forceinline__ uint16_t opA(const uint16_t *A, int lda, int ta, int M, int K, int m, int k)
{
    if (m >= M || k >= K) return 0;
    return ta ? A[(int64_t)k * lda + m] : A[(int64_t)m * lda + k];
}
__device__ __forceinline__ uint16_t opB(const uint16_t *B, int ldb, int tb, int K, int N, int k, int n)
{
    if (k >= K || n >= N) return 0;
    return tb ? B[(int64_t)n * ldb + k] : B[(int64_t)k * ldb + n];
}

// C[M][N] (+)= A(M x K) B(K x N), A(m,k) = ta ? A[k*lda+m] : A[m*lda+k],
// B(k,n) = tb ? B[n*ldb+k] : B[k*ldb+n].  One warp per 16x8 tile of C.
__global__ void __launch_bounds__(128) k_gemm_bf16(int M, int N, int K, const uint16_t *A, int lda, int ta,
                                                   const uint16_t *B, int ldb, int tb, float *C, int ldc, int acc)
{
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int ntn = (N + 7) / 8, ntm = (M + 15) / 16;
    if (warp >= ntn * ntm) return;          // uniform per warp
    const int tm = warp / ntn, tn = warp % ntn;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = tm * 16, n0 = tn * 8;
    const int rr[4] = {m0 + g, m0 + g, m0 + g + 8, m0 + g + 8};
    const int cc[4] = {n0 + 2 * t, n0 + 2 * t + 1, n0 + 2 * t, n0 + 2 * t + 1};
    float c[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        c[i] = (acc && rr[i] < M && cc[i] < N) ? C[(int64_t)rr[i] * ldc + cc[i]] : 0.0f;
    for (int k0 = 0; k0 < K; k0 += 16) {
        const int ka = k0 + 2 * t;
        uint32_t a0 = pack2(opA(A, lda, ta, M, K, m0 + g, ka), opA(A, lda, ta, M, K, m0 + g, ka + 1));
        uint32_t a1 = pack2(opA(A, lda, ta, M, K, m0 + g + 8, ka), opA(A, lda, ta, M, K, m0 + g + 8, ka + 1));
        uint32_t a2 = pack2(opA(A, lda, ta, M, K, m0 + g, ka + 8), opA(A, lda, ta, M, K, m0 + g, ka + 9));
        uint32_t a3 = pack2(opA(A, lda, ta, M, K, m0 + g + 8, ka + 8), opA(A, lda, ta, M, K, m0 + g + 8, ka + 9));
        uint32_t b0 = pack2(opB(B, ldb, tb, K, N, ka, n0 + g), opB(B, ldb, tb, K, N, ka + 1, n0 + g));
        uint32_t b1 = pack2(opB(B, ldb, tb, K, N, ka + 8, n0 + g), opB(B, ldb, tb, K, N, ka + 9, n0 + g));
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
        if (rr[i] < M && cc[i] < N) C[(int64_t)rr[i] * ldc + cc[i]] = c[i];
}

__global__ void k_to_bf16(const float *src, uint16_t *dst, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = f2bf(src[i]);
}

// H += b (per column), optional ReLU, and the BF16 copy for the next product.
__global__ void k_bias_act(float *H, const float *b, int rows, int cols, int relu, uint16_t *Hb)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)rows * cols) return;
    float v = H[i] + b[i % cols];
    if (relu) v = fmaxf(v, 0.0f);
    H[i] = v;
    if (Hb) Hb[i] = f2bf(v);
}

// dH *= [H > 0] and its BF16 copy.
__global__ void k_relu_grad(float *dH, const float *H, int64_t n, uint16_t *dHb)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float v = H[i] > 0.0f ? dH[i] : 0.0f;
    dH[i] = v;
    dHb[i] = f2bf(v);
}

// Asymmetric squared error: w (y_hat - y)^2, w = MLP_OVERSHOOT_WEIGHT if y_hat > y.
// dOut = dL/dy_hat for L = mean over rows*2 entries; per-block partial sums of w e^2.
__global__ void __launch_bounds__(256) k_loss(const float *out, const float *Y, int rows, float *dout, uint16_t *doutb,
                                              float *partial)
{
    __shared__ float red[256];
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = (int64_t)rows * MLP_OUT;
    float l = 0.0f;
    if (i < n) {
        float e = out[i] - Y[i];
        float w = e > 0.0f ? MLP_OVERSHOOT_WEIGHT : 1.0f;
        l = w * e * e;
        float gr = 2.0f * w * e / (float)n;
        dout[i] = gr;
        doutb[i] = f2bf(gr);
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// Column sums (bias gradients), one thread per column, rows in order.
__global__ void k_colsum(const float *X, int rows, int cols, float *out)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.0f;
    for (int r = 0; r < rows; ++r) s += X[(int64_t)r * cols + c];
    out[c] = s;
}

__global__ void k_adam(float *w, const float *g, float *m, float *v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2, uint16_t *wb)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    wb[i] = f2bf(wi);
}

__global__ void k_gather_rows(const float *src, const int *idx, int rows, int cols, float *dst)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)rows * cols) return;
    int r = (int)(i / cols), c = (int)(i % cols);
    dst[i] = src[(int64_t)idx[r] * cols + c];
}

unsigned blocks(int64_t n, int b) { return (unsigned)std::max<int64_t>(1, (n + b - 1) / b); }

void gemm(int M, int N, int K, const uint16_t *A, int lda, int ta, const uint16_t *B, int ldb, int tb, float *C, int ldc,
          int acc, cudaStream_t st)
{
    int64_t warps = (int64_t)((N + 7) / 8) * ((M + 15) / 16);
    k_gemm_bf16<<<blocks(warps * 32, 128), 128, 0, st>>>(M, N, K, A, lda, ta, B, ldb, tb, C, ldc, acc);
}

uint64_t splitmix64(uint64_t &s)
{
    uint64_t z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

template <class T>
cudaError_t dmalloc(T *&p, size_t n)
{
    return cudaMalloc((void **)&p, std::max<size_t>(n, 1) * sizeof(T));
}

}  // namespace

#define MLP_CU(x)                            \
    do {                                     \
        cudaError_t e_ = (x);                \
        if (e_ != cudaSuccess) return e_;    \
    } while (0)

Mlp::~Mlp()
{
    void *ps[] = {w_, wb_, g_, m_, v_, xb_, h1b_, h2b_, dob_, dh2b_, dh1b_, h1_, h2_, out_, dout_, dh2_, dh1_, lossp_,
                  xg_, yg_, idx_};
    for (void *p : ps)
        if (p) cudaFree(p);
}

cudaError_t Mlp::init(uint64_t seed, cudaStream_t st)
{
    std::vector<float> p(MLP_NPARAM, 0.0f);
    uint64_t s = seed;
    auto fill = [&](int off, int fan_out, int fan_in) {
        float a = std::sqrt(6.0f / (float)(fan_in + fan_out));
        for (int k = 0; k < fan_out * fan_in; ++k) {
            double u = (double)(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
            p[off + k] = (float)((2.0 * u - 1.0) * a);
        }
    };
    fill(OFF_W1, MLP_H, MLP_IN);
    fill(OFF_W2, MLP_H, MLP_H);
    fill(OFF_W3, MLP_OUT, MLP_H);
    return set_params(p.data(), st);
}

cudaError_t Mlp::set_params(const float *hp, cudaStream_t st)
{
    if (!w_) {
        MLP_CU(dmalloc(w_, MLP_NPARAM));
        MLP_CU(dmalloc(wb_, MLP_NPARAM));
        MLP_CU(dmalloc(g_, MLP_NPARAM));
        MLP_CU(dmalloc(m_, MLP_NPARAM));
        MLP_CU(dmalloc(v_, MLP_NPARAM));
    }
    MLP_CU(cudaMemcpyAsync(w_, hp, MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice, st));
    MLP_CU(cudaMemsetAsync(m_, 0, MLP_NPARAM * sizeof(float), st));
    MLP_CU(cudaMemsetAsync(v_, 0, MLP_NPARAM * sizeof(float), st));
    k_to_bf16<<<blocks(MLP_NPARAM, 256), 256, 0, st>>>(w_, wb_, MLP_NPARAM);
    MLP_CU(cudaGetLastError());
    MLP_CU(cudaStreamSynchronize(st));
    ready_ = true;
    return cudaSuccess;
}

cudaError_t Mlp::get_params(float *hp, cudaStream_t st)
{
    MLP_CU(cudaMemcpyAsync(hp, w_, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost, st));
    return cudaStreamSynchronize(st);
}

cudaError_t Mlp::reserve(int rows)
{
    if (rows <= cap_) return cudaSuccess;
    int cap = std::max(rows, 1024);
    void *ps[] = {xb_, h1b_, h2b_, dob_, dh2b_, dh1b_, h1_, h2_, out_, dout_, dh2_, dh1_, lossp_, xg_, yg_, idx_};
    for (void *p : ps)
        if (p) cudaFree(p);
    MLP_CU(dmalloc(xb_, (size_t)cap * MLP_IN));
    MLP_CU(dmalloc(h1b_, (size_t)cap * MLP_H));
    MLP_CU(dmalloc(h2b_, (size_t)cap * MLP_H));
    MLP_CU(dmalloc(dob_, (size_t)cap * MLP_OUT));
    MLP_CU(dmalloc(dh2b_, (size_t)cap * MLP_H));
    MLP_CU(dmalloc(dh1b_, (size_t)cap * MLP_H));
    MLP_CU(dmalloc(h1_, (size_t)cap * MLP_H));
    MLP_CU(dmalloc(h2_, (size_t)cap * MLP_H));
    MLP_CU(dmalloc(out_, (size_t)cap * MLP_OUT));
    MLP_CU(dmalloc(dout_, (size_t)cap * MLP_OUT));
    MLP_CU(dmalloc(dh2_, (size_t)cap * MLP_H));
    MLP_CU(dmalloc(dh1_, (size_t)cap * MLP_H));
    MLP_CU(dmalloc(lossp_, (size_t)cap * MLP_OUT / 256 + 2));
    MLP_CU(dmalloc(xg_, (size_t)cap * MLP_IN));
    MLP_CU(dmalloc(yg_, (size_t)cap * MLP_OUT));
    MLP_CU(dmalloc(idx_, (size_t)cap));
    cap_ = cap;
    return cudaSuccess;
}

cudaError_t Mlp::forward(const float *X, int rows, float *out, cudaStream_t st)
{
    if (!ready_) return cudaErrorNotReady;
    if (rows <= 0) return cudaSuccess;
    MLP_CU(reserve(rows));
    k_to_bf16<<<blocks((int64_t)rows * MLP_IN, 256), 256, 0, st>>>(X, xb_, (int64_t)rows * MLP_IN);
    gemm(rows, MLP_H, MLP_IN, xb_, MLP_IN, 0, wb_ + OFF_W1, MLP_IN, 1, h1_, MLP_H, 0, st);
    k_bias_act<<<blocks((int64_t)rows * MLP_H, 256), 256, 0, st>>>(h1_, w_ + OFF_B1, rows, MLP_H, 1, h1b_);
    gemm(rows, MLP_H, MLP_H, h1b_, MLP_H, 0, wb_ + OFF_W2, MLP_H, 1, h2_, MLP_H, 0, st);
    k_bias_act<<<blocks((int64_t)rows * MLP_H, 256), 256, 0, st>>>(h2_, w_ + OFF_B2, rows, MLP_H, 1, h2b_);
    gemm(rows, MLP_OUT, MLP_H, h2b_, MLP_H, 0, wb_ + OFF_W3, MLP_H, 1, out, MLP_OUT, 0, st);
    k_bias_act<<<blocks((int64_t)rows * MLP_OUT, 256), 256, 0, st>>>(out, w_ + OFF_B3, rows, MLP_OUT, 0, nullptr);
    return cudaGetLastError();
}

cudaError_t Mlp::step_batch(const float *X, const float *Y, int rows, float *loss_out, cudaStream_t st, bool update,
                            float lr, int t)
{
    MLP_CU(forward(X, rows, out_, st));
    const int64_t no = (int64_t)rows * MLP_OUT;
    const unsigned nb = blocks(no, 256);
    k_loss<<<nb, 256, 0, st>>>(out_, Y, rows, dout_, dob_, lossp_);
    // output layer
    gemm(MLP_OUT, MLP_H, rows, dob_, MLP_OUT, 1, h2b_, MLP_H, 0, g_ + OFF_W3, MLP_H, 0, st);
    k_colsum<<<1, 64, 0, st>>>(dout_, rows, MLP_OUT, g_ + OFF_B3);
    gemm(rows, MLP_H, MLP_OUT, dob_, MLP_OUT, 0, wb_ + OFF_W3, MLP_H, 0, dh2_, MLP_H, 0, st);
    k_relu_grad<<<blocks((int64_t)rows * MLP_H, 256), 256, 0, st>>>(dh2_, h2_, (int64_t)rows * MLP_H, dh2b_);
    // hidden layer 2
    gemm(MLP_H, MLP_H, rows, dh2b_, MLP_H, 1, h1b_, MLP_H, 0, g_ + OFF_W2, MLP_H, 0, st);
    k_colsum<<<1, 64, 0, st>>>(dh2_, rows, MLP_H, g_ + OFF_B2);
    gemm(rows, MLP_H, MLP_H, dh2b_, MLP_H, 0, wb_ + OFF_W2, MLP_H, 0, dh1_, MLP_H, 0, st);
    k_relu_grad<<<blocks((int64_t)rows * MLP_H, 256), 256, 0, st>>>(dh1_, h1_, (int64_t)rows * MLP_H, dh1b_);
    // hidden layer 1
    gemm(MLP_H, MLP_IN, rows, dh1b_, MLP_H, 1, xb_, MLP_IN, 0, g_ + OFF_W1, MLP_IN, 0, st);
    k_colsum<<<1, 64, 0, st>>>(dh1_, rows, MLP_H, g_ + OFF_B1);
    MLP_CU(cudaGetLastError());
    if (loss_out) {
        std::vector<float> part(nb);
        MLP_CU(cudaMemcpyAsync(part.data(), lossp_, nb * sizeof(float), cudaMemcpyDeviceToHost, st));
        MLP_CU(cudaStreamSynchronize(st));
        double s = 0.0;
        for (float p : part) s += p;
        *loss_out = (float)(s / (double)no);
    }
    if (update) {
        const float b1 = 0.9f, b2 = 0.999f;
        float c1 = 1.0f - std::pow(b1, (float)t), c2 = 1.0f - std::pow(b2, (float)t);
        k_adam<<<blocks(MLP_NPARAM, 256), 256, 0, st>>>(w_, g_, m_, v_, MLP_NPARAM, lr, b1, b2, 1e-8f, c1, c2, wb_);
        MLP_CU(cudaGetLastError());
    }
    return cudaSuccess;
}

cudaError_t Mlp::loss_grad(const float *X, const float *Y, int rows, float *loss, float *grad_host, cudaStream_t st)
{
    if (!ready_) return cudaErrorNotReady;
    MLP_CU(reserve(rows));
    MLP_CU(step_batch(X, Y, rows, loss, st, false, 0.0f, 1));
    if (grad_host) {
        MLP_CU(cudaMemcpyAsync(grad_host, g_, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost, st));
        MLP_CU(cudaStreamSynchronize(st));
    }
    return cudaSuccess;
}

cudaError_t Mlp::train(const std::vector<float> &X, const std::vector<float> &Y, int epochs, float lr, uint64_t seed,
                       float *loss, cudaStream_t st)
{
    if (!ready_) MLP_CU(init(seed, st));
    const int n = (int)(Y.size() / MLP_OUT);
    if (n <= 0) return cudaErrorInvalidValue;
    const int batch = std::min(n, 512);
    MLP_CU(reserve(batch));
    float *xall = nullptr, *yall = nullptr;
    MLP_CU(dmalloc(xall, X.size()));
    MLP_CU(dmalloc(yall, Y.size()));
    cudaError_t e = cudaMemcpyAsync(xall, X.data(), X.size() * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(yall, Y.data(), Y.size() * sizeof(float), cudaMemcpyHostToDevice, st);
    std::vector<int> perm(n);
    for (int k = 0; k < n; ++k) perm[k] = k;
    uint64_t s = seed ^ 0x5deece66dull;
    int t = 0;
    double last = 0.0;
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
        for (int k = n - 1; k > 0; --k) {               // Fisher-Yates with the seeded stream
            int j = (int)(splitmix64(s) % (uint64_t)(k + 1));
            std::swap(perm[k], perm[j]);
        }
        double acc = 0.0;
        int cnt = 0;
        for (int b0 = 0; b0 + batch <= n && e == cudaSuccess; b0 += batch) {
            e = cudaMemcpyAsync(idx_, perm.data() + b0, batch * sizeof(int), cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) break;
            k_gather_rows<<<blocks((int64_t)batch * MLP_IN, 256), 256, 0, st>>>(xall, idx_, batch, MLP_IN, xg_);
            k_gather_rows<<<blocks((int64_t)batch * MLP_OUT, 256), 256, 0, st>>>(yall, idx_, batch, MLP_OUT, yg_);
            float l = 0.0f;
            e = step_batch(xg_, yg_, batch, &l, st, true, lr, ++t);
            acc += l;
            ++cnt;
        }
        last = cnt ? acc / cnt : 0.0;
    }
    cudaStreamSynchronize(st);
    cudaFree(xall);
    cudaFree(yall);
    if (loss) *loss = (float)last;
    return e;
}

}  // namespace dem
