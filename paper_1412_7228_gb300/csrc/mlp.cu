// mlp.cu -- the learned surrogate: a 3 -> 64 -> 64 -> 4 GELU perceptron in
// FP32 with hand-written training (forward, backward, Adam) and inference
// kernels, and a batched bisection that inverts sigma(kappa).
//
// Training works on chunks of kChunk samples per CTA: one thread per sample
// runs the forward and backward pass, keeping activations and
// pre-activation gradients of the chunk in shared memory; the CTA then forms
// its share of every weight gradient (sums over its samples) and writes them
// as one row of partial gradients.  k_reduce_adam adds the rows in a fixed
// order (deterministic) and applies Adam.  The matrices are 64 wide and the
// data set a few thousand samples, so plain FP32 FMAs are used (FP32
// accumulation is required; tensor cores would round the operands).
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "lbm_internal.cuh"

namespace {

constexpr int NI = LBM_MLP_IN, NH = LBM_MLP_HIDDEN, NO = LBM_MLP_OUT;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NI, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NO * NH, NP = OFF_B3 + NO;
static_assert(NP == LBM_MLP_NPARAMS, "parameter count");
constexpr int kChunk = 64;          // samples per CTA in the training kernel
constexpr int kThreads = 128;
constexpr int kStride = NH + 1;     // padded row of a per-sample activation vector
constexpr int NPL = NP + 1;         // partial-gradient row: parameters + loss

struct Norm {
    float in_mean[NI], in_std[NI], out_mean[NO], out_std[NO];
};

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// ---- training: forward + backward of a chunk, partial gradients ----------
// X: n x 3 standardised inputs, Y: n x 4 standardised targets, idx: sample
// order (minibatch = idx[first .. first + count)).  inv_norm = 1 / (count * 4).
__global__ void __launch_bounds__(kThreads) k_grad(const float* __restrict__ P, const float* __restrict__ X,
                                                   const float* __restrict__ Y, const int* __restrict__ idx, int first,
                                                   int count, float inv_norm, float* __restrict__ partials) {
    extern __shared__ float sm[];
    float* W = sm;                               // NP parameters
    float* H1 = W + ((NP + 31) / 32) * 32;       // kChunk x kStride
    float* H2 = H1 + kChunk * kStride;
    float* D1 = H2 + kChunk * kStride;           // dZ1
    float* D2 = D1 + kChunk * kStride;           // dZ2
    float* DY = D2 + kChunk * kStride;           // kChunk x NO
    float* XS = DY + kChunk * NO;                // kChunk x NI
    float* LS = XS + kChunk * NI;                // kChunk losses
    const int tid = threadIdx.x;
    for (int p = tid; p < NP; p += kThreads) W[p] = P[p];
    const int c0 = blockIdx.x * kChunk;
    const int nloc = min(kChunk, count - c0);
    __syncthreads();

    for (int s = tid; s < kChunk; s += kThreads) {
        if (s >= nloc) {   // pad rows contribute nothing
            for (int j = 0; j < NH; ++j) H1[s * kStride + j] = H2[s * kStride + j] = D1[s * kStride + j] =
                D2[s * kStride + j] = 0.0f;
            for (int k = 0; k < NO; ++k) DY[s * NO + k] = 0.0f;
            for (int c = 0; c < NI; ++c) XS[s * NI + c] = 0.0f;
            LS[s] = 0.0f;
            continue;
        }
        const int g = idx[first + c0 + s];
        float x[NI];
        for (int c = 0; c < NI; ++c) XS[s * NI + c] = x[c] = X[g * NI + c];
        float* h1 = H1 + s * kStride;
        float* d1 = D1 + s * kStride;   // holds z1 until the backward pass overwrites it
        for (int j = 0; j < NH; ++j) {
            float z = W[OFF_B1 + j];
            for (int c = 0; c < NI; ++c) z = fmaf(W[OFF_W1 + j * NI + c], x[c], z);
            d1[j] = z;
            h1[j] = gelu(z);
        }
        float y[NO];
        for (int k = 0; k < NO; ++k) y[k] = W[OFF_B3 + k];
        float* h2 = H2 + s * kStride;
        float* d2 = D2 + s * kStride;   // holds z2 until the backward pass overwrites it
        for (int j = 0; j < NH; ++j) {
            float z = W[OFF_B2 + j];
            for (int i = 0; i < NH; ++i) z = fmaf(W[OFF_W2 + j * NH + i], h1[i], z);
            d2[j] = z;
            const float h = gelu(z);
            h2[j] = h;
            for (int k = 0; k < NO; ++k) y[k] = fmaf(W[OFF_W3 + k * NH + j], h, y[k]);
        }
        float loss = 0.0f, dy[NO];
        for (int k = 0; k < NO; ++k) {
            const float e = y[k] - Y[g * NO + k];
            loss = fmaf(e, e, loss);
            dy[k] = 2.0f * e * inv_norm;
            DY[s * NO + k] = dy[k];
        }
        LS[s] = loss;
        // dZ2 = (W3^T dY) * gelu'(z2)
        for (int j = 0; j < NH; ++j) {
            float dh = 0.0f;
            for (int k = 0; k < NO; ++k) dh = fmaf(W[OFF_W3 + k * NH + j], dy[k], dh);
            d2[j] = dh * gelu_d(d2[j]);
        }
        // dZ1 = (W2^T dZ2) * gelu'(z1)
        for (int i = 0; i < NH; ++i) {
            float dh = 0.0f;
            for (int j = 0; j < NH; ++j) dh = fmaf(W[OFF_W2 + j * NH + i], d2[j], dh);
            d1[i] = dh * gelu_d(d1[i]);
        }
    }
    __syncthreads();

    // this chunk's share of every gradient entry, summed over its samples
    float* out = partials + static_cast<long long>(blockIdx.x) * NPL;
    for (int p = tid; p < NP; p += kThreads) {
        float acc = 0.0f;
        if (p < OFF_B1) {                                   // dW1[j][c] = sum dZ1[s][j] x[s][c]
            const int j = p / NI, c = p % NI;
            for (int s = 0; s < kChunk; ++s) acc = fmaf(D1[s * kStride + j], XS[s * NI + c], acc);
        } else if (p < OFF_W2) {                            // db1
            const int j = p - OFF_B1;
            for (int s = 0; s < kChunk; ++s) acc += D1[s * kStride + j];
        } else if (p < OFF_B2) {                            // dW2[j][i] = sum dZ2[s][j] h1[s][i]
            const int j = (p - OFF_W2) / NH, i = (p - OFF_W2) % NH;
            for (int s = 0; s < kChunk; ++s) acc = fmaf(D2[s * kStride + j], H1[s * kStride + i], acc);
        } else if (p < OFF_W3) {                            // db2
            const int j = p - OFF_B2;
            for (int s = 0; s < kChunk; ++s) acc += D2[s * kStride + j];
        } else if (p < OFF_B3) {                            // dW3[k][j] = sum dY[s][k] h2[s][j]
            const int k = (p - OFF_W3) / NH, j = (p - OFF_W3) % NH;
            for (int s = 0; s < kChunk; ++s) acc = fmaf(DY[s * NO + k], H2[s * kStride + j], acc);
        } else {                                            // db3
            const int k = p - OFF_B3;
            for (int s = 0; s < kChunk; ++s) acc += DY[s * NO + k];
        }
        out[p] = acc;
    }
    if (tid == 0) {
        float l = 0.0f;
        for (int s = 0; s < kChunk; ++s) l += LS[s];
        out[NP] = l * inv_norm;
    }
}

size_t grad_smem() {
    return sizeof(float) * (((NP + 31) / 32) * 32 + 4 * kChunk * kStride + kChunk * NO + kChunk * NI + kChunk);
}

// Sum the partial-gradient rows in a fixed order; optionally apply Adam.
__global__ void k_reduce_adam(const float* __restrict__ partials, int nparts, float* __restrict__ P,
                              float* __restrict__ M, float* __restrict__ V, float* __restrict__ grad_out,
                              float* __restrict__ loss_out, int do_update, float lr, float b1, float b2, float eps,
                              float c1, float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > NP) return;
    float g = 0.0f;
    for (int r = 0; r < nparts; ++r) g += partials[static_cast<long long>(r) * NPL + p];
    if (p == NP) {
        if (loss_out) *loss_out = g;
        return;
    }
    if (grad_out) grad_out[p] = g;
    if (do_update) {
        const float m = b1 * M[p] + (1.0f - b1) * g;
        const float v = b2 * V[p] + (1.0f - b2) * g * g;
        M[p] = m;
        V[p] = v;
        P[p] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

__device__ void forward_one(const float* W, const float (&x)[NI], float (&y)[NO]) {
    float h1[NH];
    for (int j = 0; j < NH; ++j) {
        float z = W[OFF_B1 + j];
        for (int c = 0; c < NI; ++c) z = fmaf(W[OFF_W1 + j * NI + c], x[c], z);
        h1[j] = gelu(z);
    }
    for (int k = 0; k < NO; ++k) y[k] = W[OFF_B3 + k];
    for (int j = 0; j < NH; ++j) {
        float z = W[OFF_B2 + j];
        for (int i = 0; i < NH; ++i) z = fmaf(W[OFF_W2 + j * NH + i], h1[i], z);
        const float h = gelu(z);
        for (int k = 0; k < NO; ++k) y[k] = fmaf(W[OFF_W3 + k * NH + j], h, y[k]);
    }
}

// Inference on raw inputs: standardise, forward, de-standardise.
__global__ void __launch_bounds__(kThreads) k_predict(const float* __restrict__ P, Norm nm,
                                                      const float* __restrict__ X, int n, float* __restrict__ Y) {
    __shared__ float W[NP];
    for (int p = threadIdx.x; p < NP; p += blockDim.x) W[p] = P[p];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float x[NI], y[NO];
    for (int c = 0; c < NI; ++c) x[c] = (X[s * NI + c] - nm.in_mean[c]) / nm.in_std[c];
    forward_one(W, x, y);
    for (int k = 0; k < NO; ++k) Y[s * NO + k] = y[k] * nm.out_std[k] + nm.out_mean[k];
}

// Bisection on kappa for each target: predicted sigma (output 0) decreases in kappa.
__global__ void __launch_bounds__(kThreads) k_invert(const float* __restrict__ P, Norm nm,
                                                     const float* __restrict__ tr, const float* __restrict__ A,
                                                     const float* __restrict__ sig, int m, float lo, float hi,
                                                     float* __restrict__ kappa) {
    __shared__ float W[NP];
    for (int p = threadIdx.x; p < NP; p += blockDim.x) W[p] = P[p];
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    auto sigma_at = [&](float k) {
        float x[NI] = {(tr[t] - nm.in_mean[0]) / nm.in_std[0], (A[t] - nm.in_mean[1]) / nm.in_std[1],
                       (k - nm.in_mean[2]) / nm.in_std[2]};
        float y[NO];
        forward_one(W, x, y);
        return y[0] * nm.out_std[0] + nm.out_mean[0];
    };
    const float target = sig[t];
    float a = lo, b = hi;
    float fa = sigma_at(a) - target, fb = sigma_at(b) - target;
    if (!(fa >= 0.0f && fb <= 0.0f)) {
        kappa[t] = nanf("");
        return;
    }
    for (int it = 0; it < 40; ++it) {
        const float mid = 0.5f * (a + b);
        const float fm = sigma_at(mid) - target;
        if (fm >= 0.0f) a = mid; else b = mid;
    }
    kappa[t] = 0.5f * (a + b);
}

uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double uniform01(uint64_t& s) { return (splitmix(s) >> 11) * (1.0 / 9007199254740992.0); }

}  // namespace

struct lbm_mlp {
    int max_n = 0;
    cudaStream_t st = nullptr;
    Norm norm{};
    float *P = nullptr, *M = nullptr, *V = nullptr, *X = nullptr, *Y = nullptr, *partials = nullptr,
          *grad = nullptr, *loss = nullptr, *io = nullptr;
    int* idx = nullptr;
    int adam_t = 0;
};

namespace {

bool valid(lbm_mlp* m) { return m && m->P; }

int standardise_upload(lbm_mlp* m, const float* X, const float* Y, int n) {
    std::vector<float> xs(static_cast<size_t>(n) * NI), ys(static_cast<size_t>(n) * NO);
    for (int s = 0; s < n; ++s) {
        for (int c = 0; c < NI; ++c) xs[s * NI + c] = (X[s * NI + c] - m->norm.in_mean[c]) / m->norm.in_std[c];
        for (int k = 0; k < NO; ++k) ys[s * NO + k] = (Y[s * NO + k] - m->norm.out_mean[k]) / m->norm.out_std[k];
    }
    if (cudaMemcpyAsync(m->X, xs.data(), xs.size() * sizeof(float), cudaMemcpyHostToDevice, m->st) != cudaSuccess ||
        cudaMemcpyAsync(m->Y, ys.data(), ys.size() * sizeof(float), cudaMemcpyHostToDevice, m->st) != cudaSuccess ||
        cudaStreamSynchronize(m->st) != cudaSuccess)
        return LBM_ECUDA;
    return LBM_OK;
}

int set_order(lbm_mlp* m, const std::vector<int>& order) {
    if (cudaMemcpyAsync(m->idx, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice, m->st) !=
            cudaSuccess ||
        cudaStreamSynchronize(m->st) != cudaSuccess)
        return LBM_ECUDA;
    return LBM_OK;
}

// gradient (and optional Adam update) over idx[first .. first+count)
cudaError_t grad_pass(lbm_mlp* m, int first, int count, bool update, float lr, float b1, float b2, float eps,
                      float* loss_slot) {
    const int chunks = (count + kChunk - 1) / kChunk;
    k_grad<<<chunks, kThreads, grad_smem(), m->st>>>(m->P, m->X, m->Y, m->idx, first, count,
                                                      1.0f / (static_cast<float>(count) * NO), m->partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    float c1 = 1.0f, c2 = 1.0f;
    if (update) {
        ++m->adam_t;
        c1 = 1.0f - std::pow(b1, static_cast<float>(m->adam_t));
        c2 = 1.0f - std::pow(b2, static_cast<float>(m->adam_t));
    }
    k_reduce_adam<<<(NP + 1 + 255) / 256, 256, 0, m->st>>>(m->partials, chunks, m->P, m->M, m->V, m->grad, loss_slot,
                                                           update ? 1 : 0, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

int lbm_mlp_create(lbm_mlp** out, int max_samples, unsigned long long seed, void* stream) {
    if (!out || max_samples < 1) return LBM_EINVAL;
    *out = nullptr;
    lbm_mlp* m = new lbm_mlp();
    m->max_n = max_samples;
    m->st = static_cast<cudaStream_t>(stream);
    const int max_chunks = (max_samples + kChunk - 1) / kChunk;
    const size_t pbytes = NP * sizeof(float);
    bool ok = cudaMalloc(&m->P, pbytes) == cudaSuccess && cudaMalloc(&m->M, pbytes) == cudaSuccess &&
              cudaMalloc(&m->V, pbytes) == cudaSuccess && cudaMalloc(&m->grad, pbytes) == cudaSuccess &&
              cudaMalloc(&m->loss, 4096 * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->X, sizeof(float) * NI * max_samples) == cudaSuccess &&
              cudaMalloc(&m->Y, sizeof(float) * NO * max_samples) == cudaSuccess &&
              cudaMalloc(&m->io, sizeof(float) * NO * max_samples) == cudaSuccess &&
              cudaMalloc(&m->idx, sizeof(int) * max_samples) == cudaSuccess &&
              cudaMalloc(&m->partials, sizeof(float) * NPL * static_cast<size_t>(max_chunks)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        lbm_mlp_destroy(m);
        return LBM_ENOMEM;
    }
    if (cudaFuncSetAttribute(k_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(grad_smem())) !=
        cudaSuccess) {
        lbm_mlp_destroy(m);
        return LBM_ECUDA;
    }
    // Glorot-uniform weights from a seeded splitmix64 stream, zero biases
    std::vector<float> p(NP, 0.0f);
    uint64_t s = seed;
    auto fill = [&](int off, int rows, int cols) {
        const double a = std::sqrt(6.0 / (rows + cols));
        for (int i = 0; i < rows * cols; ++i) p[off + i] = static_cast<float>((2.0 * uniform01(s) - 1.0) * a);
    };
    fill(OFF_W1, NH, NI);
    fill(OFF_W2, NH, NH);
    fill(OFF_W3, NO, NH);
    for (int c = 0; c < NI; ++c) { m->norm.in_mean[c] = 0.0f; m->norm.in_std[c] = 1.0f; }
    for (int k = 0; k < NO; ++k) { m->norm.out_mean[k] = 0.0f; m->norm.out_std[k] = 1.0f; }
    int rc = lbm_mlp_set_params(m, p.data());
    if (rc) {
        lbm_mlp_destroy(m);
        return rc;
    }
    *out = m;
    return LBM_OK;
}

void lbm_mlp_destroy(lbm_mlp* m) {
    if (!m) return;
    if (m->P) cudaStreamSynchronize(m->st);
    float* bufs[] = {m->P, m->M, m->V, m->X, m->Y, m->partials, m->grad, m->loss, m->io};
    for (float* b : bufs)
        if (b) cudaFree(b);
    if (m->idx) cudaFree(m->idx);
    delete m;
}

int lbm_mlp_set_normalization(lbm_mlp* m, const float in_mean[3], const float in_std[3], const float out_mean[4],
                              const float out_std[4]) {
    if (!valid(m) || !in_mean || !in_std || !out_mean || !out_std) return LBM_EINVAL;
    for (int c = 0; c < NI; ++c)
        if (!(in_std[c] > 0.0f) || !std::isfinite(in_mean[c])) return LBM_EINVAL;
    for (int k = 0; k < NO; ++k)
        if (!(out_std[k] > 0.0f) || !std::isfinite(out_mean[k])) return LBM_EINVAL;
    std::memcpy(m->norm.in_mean, in_mean, sizeof m->norm.in_mean);
    std::memcpy(m->norm.in_std, in_std, sizeof m->norm.in_std);
    std::memcpy(m->norm.out_mean, out_mean, sizeof m->norm.out_mean);
    std::memcpy(m->norm.out_std, out_std, sizeof m->norm.out_std);
    return LBM_OK;
}

int lbm_mlp_set_params(lbm_mlp* m, const float* params) {
    if (!valid(m) || !params) return LBM_EINVAL;
    if (cudaMemcpyAsync(m->P, params, NP * sizeof(float), cudaMemcpyHostToDevice, m->st) != cudaSuccess ||
        cudaMemsetAsync(m->M, 0, NP * sizeof(float), m->st) != cudaSuccess ||
        cudaMemsetAsync(m->V, 0, NP * sizeof(float), m->st) != cudaSuccess ||
        cudaStreamSynchronize(m->st) != cudaSuccess)
        return LBM_ECUDA;
    m->adam_t = 0;
    return LBM_OK;
}

int lbm_mlp_get_params(lbm_mlp* m, float* params) {
    if (!valid(m) || !params) return LBM_EINVAL;
    if (cudaMemcpyAsync(params, m->P, NP * sizeof(float), cudaMemcpyDeviceToHost, m->st) != cudaSuccess ||
        cudaStreamSynchronize(m->st) != cudaSuccess)
        return LBM_ECUDA;
    return LBM_OK;
}

int lbm_mlp_loss_grad(lbm_mlp* m, const float* X, const float* Y, int n, float* loss, float* grad) {
    if (!valid(m) || !X || !Y || n < 1 || n > m->max_n) return LBM_EINVAL;
    int rc = standardise_upload(m, X, Y, n);
    if (rc) return rc;
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    if ((rc = set_order(m, order))) return rc;
    if (grad_pass(m, 0, n, false, 0, 0, 0, 0, m->loss) != cudaSuccess) return LBM_ECUDA;
    if (loss && cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->st) != cudaSuccess)
        return LBM_ECUDA;
    if (grad && cudaMemcpyAsync(grad, m->grad, NP * sizeof(float), cudaMemcpyDeviceToHost, m->st) != cudaSuccess)
        return LBM_ECUDA;
    return cudaStreamSynchronize(m->st) == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

int lbm_mlp_adam_step(lbm_mlp* m, const float* X, const float* Y, int n, float lr, float beta1, float beta2,
                      float eps) {
    if (!valid(m) || !X || !Y || n < 1 || n > m->max_n || !(lr > 0)) return LBM_EINVAL;
    int rc = standardise_upload(m, X, Y, n);
    if (rc) return rc;
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    if ((rc = set_order(m, order))) return rc;
    if (grad_pass(m, 0, n, true, lr, beta1, beta2, eps, m->loss) != cudaSuccess) return LBM_ECUDA;
    return cudaStreamSynchronize(m->st) == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

int lbm_mlp_train(lbm_mlp* m, const float* X, const float* Y, int n, int epochs, int batch, float lr,
                  unsigned long long seed, float* loss_per_epoch) {
    if (!valid(m) || !X || !Y || n < 1 || n > m->max_n || epochs < 1 || batch < 1 || !(lr > 0)) return LBM_EINVAL;
    int rc = standardise_upload(m, X, Y, n);
    if (rc) return rc;
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    uint64_t s = seed;
    const int nb = (n + batch - 1) / batch;
    std::vector<float> losses(nb);
    for (int e = 0; e < epochs; ++e) {
        for (int i = n - 1; i > 0; --i) {   // Fisher-Yates with splitmix64
            const int j = static_cast<int>(splitmix(s) % static_cast<uint64_t>(i + 1));
            std::swap(order[i], order[j]);
        }
        if ((rc = set_order(m, order))) return rc;
        for (int b = 0; b < nb; ++b) {
            const int first = b * batch, count = std::min(batch, n - first);
            if (grad_pass(m, first, count, true, lr, 0.9f, 0.999f, 1e-8f, m->loss + (b % 4096)) != cudaSuccess)
                return LBM_ECUDA;
        }
        if (loss_per_epoch) {
            const int k = std::min(nb, 4096);
            if (cudaMemcpyAsync(losses.data(), m->loss, k * sizeof(float), cudaMemcpyDeviceToHost, m->st) !=
                    cudaSuccess ||
                cudaStreamSynchronize(m->st) != cudaSuccess)
                return LBM_ECUDA;
            double acc = 0;
            for (int b = 0; b < k; ++b) acc += losses[b];
            loss_per_epoch[e] = static_cast<float>(acc / k);
        }
    }
    return cudaStreamSynchronize(m->st) == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

int lbm_mlp_predict(lbm_mlp* m, const float* X, int n, float* Y) {
    if (!valid(m) || !X || !Y || n < 1 || n > m->max_n) return LBM_EINVAL;
    if (cudaMemcpyAsync(m->X, X, sizeof(float) * NI * n, cudaMemcpyHostToDevice, m->st) != cudaSuccess)
        return LBM_ECUDA;
    k_predict<<<(n + kThreads - 1) / kThreads, kThreads, 0, m->st>>>(m->P, m->norm, m->X, n, m->io);
    if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
    if (cudaMemcpyAsync(Y, m->io, sizeof(float) * NO * n, cudaMemcpyDeviceToHost, m->st) != cudaSuccess ||
        cudaStreamSynchronize(m->st) != cudaSuccess)
        return LBM_ECUDA;
    return LBM_OK;
}

int lbm_mlp_invert_kappa(lbm_mlp* m, const float* t_over_tc, const float* A, const float* sigma, int count,
                         float kappa_lo, float kappa_hi, float* kappa_out) {
    if (!valid(m) || !t_over_tc || !A || !sigma || !kappa_out || count < 1 || count > m->max_n ||
        !(kappa_lo < kappa_hi))
        return LBM_EINVAL;
    // inputs in m->X (3 columns reused as t, A, sigma), kappas out in m->io
    std::vector<float> packed(static_cast<size_t>(count) * 3);
    for (int i = 0; i < count; ++i) {
        packed[i] = t_over_tc[i];
        packed[count + i] = A[i];
        packed[2 * count + i] = sigma[i];
    }
    if (cudaMemcpyAsync(m->X, packed.data(), packed.size() * sizeof(float), cudaMemcpyHostToDevice, m->st) !=
        cudaSuccess)
        return LBM_ECUDA;
    k_invert<<<(count + kThreads - 1) / kThreads, kThreads, 0, m->st>>>(m->P, m->norm, m->X, m->X + count,
                                                                      m->X + 2 * count, count, kappa_lo, kappa_hi,
                                                                      m->io);
    if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
    if (cudaMemcpyAsync(kappa_out, m->io, sizeof(float) * count, cudaMemcpyDeviceToHost, m->st) != cudaSuccess ||
        cudaStreamSynchronize(m->st) != cudaSuccess)
        return LBM_ECUDA;
    return LBM_OK;
}

}  // extern "C"
