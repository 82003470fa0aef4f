// mlp.cuh -- the learned cost model's network and its training step, as
// CUDA kernels (FP32): F -> H -> H -> 1 with ReLU,
//   h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = w3 . h2 + b3,
//   loss = mean_b (y_b - t_b)^2, relu'(0) = 0,
// trained with Adam (Kingma and Ba, 2015).  It predicts the log run time
// of a kernel instantiation from its features, the "profiling information ...
// to guide more-advanced autotuning" of the paper's future work (Sec. 6).
//
// Parameters are one flat FP32 vector in the order W1[H][F], b1[H],
// W2[H][H], b2[H], w3[H], b3 (row-major, output index slowest).
// Gradients are summed per block into partial vectors and reduced in a fixed
// block order, so a training step is deterministic.
#ifndef CJ_MLP_CUH
#define CJ_MLP_CUH

namespace cj {

template <int H>
struct MlpLayout {
    int F;
    __host__ __device__ int w1() const { return 0; }
    __host__ __device__ int b1() const { return H * F; }
    __host__ __device__ int w2() const { return H * F + H; }
    __host__ __device__ int b2() const { return H * F + H + H * H; }
    __host__ __device__ int w3() const { return H * F + H + H * H + H; }
    __host__ __device__ int b3() const { return H * F + H + H * H + 2 * H; }
    __host__ __device__ int count() const { return H * F + H + H * H + 2 * H + 1; }
};

// Forward pass, one thread per sample; the parameters sit in shared memory.
template <int H>
__global__ void __launch_bounds__(128)
mlp_forward(const float* __restrict__ theta, const float* __restrict__ X, float* __restrict__ y, int F,
            long long B) {
    extern __shared__ __align__(16) float sp[];
    const MlpLayout<H> L{F};
    for (int i = threadIdx.x; i < L.count(); i += blockDim.x) sp[i] = theta[i];
    __syncthreads();
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float* x = X + b * F;
    float h1[H];
#pragma unroll
    for (int o = 0; o < H; ++o) {
        float s = sp[L.b1() + o];
        for (int i = 0; i < F; ++i) s = __fmaf_rn(sp[L.w1() + o * F + i], x[i], s);
        h1[o] = s > 0.f ? s : 0.f;
    }
    float out = sp[L.b3()];
    for (int o = 0; o < H; ++o) {
        float s = sp[L.b2() + o];
#pragma unroll
        for (int i = 0; i < H; ++i) s = __fmaf_rn(sp[L.w2() + o * H + i], h1[i], s);
        const float h2 = s > 0.f ? s : 0.f;
        out = __fmaf_rn(sp[L.w3() + o], h2, out);
    }
    y[b] = out;
}

// Loss and gradient of one block of BS samples: forward, then backward with
// the activations kept in shared memory; writes this block's partial
// gradient (count() floats) and partial squared-error sum.
// Shared memory: params | X[BS][F] | H1[BS][H] | D2[BS][H] | D1[BS][H] |
// DY[BS] | SQ[BS].
template <int H, int BS>
__global__ void __launch_bounds__(BS)
mlp_grad_partial(const float* __restrict__ theta, const float* __restrict__ X, const float* __restrict__ t,
                 int F, long long B, float* __restrict__ partial, float* __restrict__ partial_loss) {
    extern __shared__ __align__(16) float sm[];
    const MlpLayout<H> L{F};
    const int P = L.count();
    float* sp = sm;
    float* sx = sp + ((P + 3) & ~3);
    float* sh1 = sx + BS * F;
    float* sd2 = sh1 + BS * H;
    float* sd1 = sd2 + BS * H;
    float* sdy = sd1 + BS * H;
    float* ssq = sdy + BS;
    const int tid = threadIdx.x;
    for (int i = tid; i < P; i += BS) sp[i] = theta[i];
    const long long b0 = (long long)blockIdx.x * BS;
    const int nb = (B - b0) < BS ? (int)(B - b0) : BS;
    for (int i = tid; i < BS * F; i += BS) sx[i] = i < nb * F ? X[b0 * F + i] : 0.f;
    __syncthreads();
    sdy[tid] = 0.f;
    ssq[tid] = 0.f;
    if (tid < nb) {
        const float* x = sx + tid * F;
        float* h1 = sh1 + tid * H;
        for (int o = 0; o < H; ++o) {
            float s = sp[L.b1() + o];
            for (int i = 0; i < F; ++i) s = __fmaf_rn(sp[L.w1() + o * F + i], x[i], s);
            h1[o] = s > 0.f ? s : 0.f;   // h1 > 0 exactly where z1 > 0
        }
        float* d2 = sd2 + tid * H;
        float* h2 = sd1 + tid * H;       // D1 holds h2 until the w3 gradient is taken
        float y = sp[L.b3()];
        for (int o = 0; o < H; ++o) {
            float s = sp[L.b2() + o];
            for (int i = 0; i < H; ++i) s = __fmaf_rn(sp[L.w2() + o * H + i], h1[i], s);
            h2[o] = s > 0.f ? s : 0.f;
            d2[o] = s;                   // z2 for now
            y = __fmaf_rn(sp[L.w3() + o], h2[o], y);
        }
        const float r = y - t[b0 + tid];
        const float dy = 2.f * r / (float)B;
        ssq[tid] = r * r;
        sdy[tid] = dy;
        for (int o = 0; o < H; ++o) d2[o] = d2[o] > 0.f ? dy * sp[L.w3() + o] : 0.f;   // dloss/dz2
    }
    __syncthreads();
    float* pg = partial + (long long)blockIdx.x * P;
    for (int o = tid; o < H; o += BS) {
        float s = 0.f;
        for (int k = 0; k < nb; ++k) s = __fmaf_rn(sdy[k], sd1[k * H + o], s);
        pg[L.w3() + o] = s;
    }
    if (tid == 0) {
        float g = 0.f, l = 0.f;
        for (int k = 0; k < nb; ++k) {
            g += sdy[k];
            l += ssq[k];
        }
        pg[L.b3()] = g;
        partial_loss[blockIdx.x] = l;
    }
    __syncthreads();
    // D1 <- dloss/dz1 = relu'(z1) * (W2^T d2)
    if (tid < nb) {
        const float* d2 = sd2 + tid * H;
        const float* h1 = sh1 + tid * H;
        float* d1 = sd1 + tid * H;
        for (int i = 0; i < H; ++i) {
            float s = 0.f;
            for (int o = 0; o < H; ++o) s = __fmaf_rn(sp[L.w2() + o * H + i], d2[o], s);
            d1[i] = h1[i] > 0.f ? s : 0.f;
        }
    }
    __syncthreads();
    for (int e = tid; e < H * H; e += BS) {    // W2: sum_k d2[k][o] h1[k][i]
        const int o = e / H, i = e - o * H;
        float s = 0.f;
        for (int k = 0; k < nb; ++k) s = __fmaf_rn(sd2[k * H + o], sh1[k * H + i], s);
        pg[L.w2() + e] = s;
    }
    for (int o = tid; o < H; o += BS) {
        float s2 = 0.f, s1 = 0.f;
        for (int k = 0; k < nb; ++k) {
            s2 += sd2[k * H + o];
            s1 += sd1[k * H + o];
        }
        pg[L.b2() + o] = s2;
        pg[L.b1() + o] = s1;
    }
    for (int e = tid; e < H * F; e += BS) {    // W1: sum_k d1[k][o] x[k][i]
        const int o = e / F, i = e - o * F;
        float s = 0.f;
        for (int k = 0; k < nb; ++k) s = __fmaf_rn(sd1[k * H + o], sx[k * F + i], s);
        pg[L.w1() + e] = s;
    }
}

// Sum the partial gradients over blocks (fixed order) and apply one Adam
// step; also writes the summed gradient and the mean loss.
__global__ void __launch_bounds__(256)
mlp_reduce_adam(const float* __restrict__ partial, const float* __restrict__ partial_loss, int nblocks, int P,
                float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                float* __restrict__ grad_out, float* __restrict__ loss_out, long long B, int step, float lr,
                float beta1, float beta2, float eps, int apply) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0 && loss_out) {
        double l = 0.0;
        for (int k = 0; k < nblocks; ++k) l += partial_loss[k];
        *loss_out = (float)(l / (double)B);
    }
    if (p >= P) return;
    float g = 0.f;
    for (int k = 0; k < nblocks; ++k) g += partial[(long long)k * P + p];
    if (grad_out) grad_out[p] = g;
    if (!apply) return;
    const float mk = beta1 * m[p] + (1.f - beta1) * g;
    const float vk = beta2 * v[p] + (1.f - beta2) * g * g;
    m[p] = mk;
    v[p] = vk;
    const float c1 = 1.f - powf(beta1, (float)step);
    const float c2 = 1.f - powf(beta2, (float)step);
    theta[p] = theta[p] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

}  // namespace cj
#endif
