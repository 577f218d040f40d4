// rankmlp.cu — learned ACA rank predictor (not part of the paper).
//
// A small MLP maps the geometry of an admissible block to its expected ACA
// rank; the build uses the prediction only to size each block's ACA
// workspace and to group blocks of similar size into batches.  The ACA's own
// stopping test still decides the rank, and a block whose rank exceeds its
// predicted capacity is re-run with a larger one, so the prediction never
// changes the result.  The rank grows with k_s diam (Sec. 5.3, Sec. 8), hence
// the features:
//   f = (k_s D, k_p D, dist/D, log2|tau|, log2|sigma|, log10 eps),
//   D = max(diam_box tau, diam_box sigma), dist = dist_box (Sec. 6.1),
// standardised with the training set's mean and deviation; the target is
// log(1 + rank/3) (rank-3 steps), also standardised.
// Network: 6 -> 64 -> 64 -> 1, exact GELU, FP32.  Training: mean squared
// error, Adam, mini-batches drawn by a counter-based hash of (seed, step, i).
//
// Parameter block (HM_RANK_MODEL_PARAMS floats):
//   [0,6) feature mean, [6,12) feature deviation, 12 target mean, 13 target
//   deviation, then W1 (64 x 6, row-major), b1 (64), W2 (64 x 64), b2 (64),
//   w3 (64), b3 (1).
#include <cmath>
#include <vector>

#include "hm_internal.h"

namespace {

constexpr int NF = 6, NH = 64;
constexpr int OFF_W1 = 14, OFF_B1 = OFF_W1 + NH * NF, OFF_W2 = OFF_B1 + NH,
              OFF_B2 = OFF_W2 + NH * NH, OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH,
              NPARAM = OFF_B3 + 1;
static_assert(NPARAM == HM_RANK_MODEL_PARAMS, "parameter layout");
constexpr int NW = NPARAM - OFF_W1;  // trainable parameters

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118f)); }
__device__ __forceinline__ float gelu_d(float z) {
    return 0.5f * (1.f + erff(z * 0.70710678118f)) + z * 0.39894228040f * expf(-0.5f * z * z);
}

// Z = A W^T + b, H = GELU(Z): A (B x K), W (N x K), one thread per output.
__global__ void dense_fwd_kernel(const float* A, int K, const float* W, const float* b, int N,
                                 int64_t B, float* Z, float* H) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= B * N) return;
    const int64_t i = q / N;
    const int j = (int)(q - i * N);
    float z = b[j];
    for (int k = 0; k < K; ++k) z = fmaf(A[i * K + k], W[j * K + k], z);
    Z[q] = z;
    if (H) H[q] = gelu(z);
}

// standardised features of the selected samples (batch index list or all)
__global__ void gather_std_kernel(const float* F, const float* tgt, const float* P,
                                  const int64_t* idx, int64_t B, float* X, float* Y) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= B) return;
    const int64_t s = idx ? idx[i] : i;
    for (int f = 0; f < NF; ++f) X[i * NF + f] = (F[s * NF + f] - P[f]) / P[NF + f];
    if (tgt && Y) Y[i] = (tgt[s] - P[12]) / P[13];
}

// out = H2 w3 + b3; dout = 2 (out - y) / B (or plain output when y is null)
__global__ void head_kernel(const float* H2, const float* P, const float* Y, int64_t B, float* out,
                            float* dout) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= B) return;
    float o = P[OFF_B3];
    for (int k = 0; k < NH; ++k) o = fmaf(H2[i * NH + k], P[OFF_W3 + k], o);
    out[i] = o;
    if (Y) dout[i] = 2.f * (o - Y[i]) / (float)B;
}

// dZ2 = dout w3 o GELU'(Z2)
__global__ void back_head_kernel(const float* dout, const float* P, const float* Z2, int64_t B,
                                 float* dZ2) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= B * NH) return;
    const int64_t i = q / NH;
    const int j = (int)(q - i * NH);
    dZ2[q] = dout[i] * P[OFF_W3 + j] * gelu_d(Z2[q]);
}

// dZ1 = (dZ2 W2) o GELU'(Z1)
__global__ void back_hidden_kernel(const float* dZ2, const float* P, const float* Z1, int64_t B,
                                   float* dZ1) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= B * NH) return;
    const int64_t i = q / NH;
    const int k = (int)(q - i * NH);
    float s = 0.f;
    for (int j = 0; j < NH; ++j) s = fmaf(dZ2[i * NH + j], P[OFF_W2 + j * NH + k], s);
    dZ1[q] = s * gelu_d(Z1[q]);
}

// gradient of every trainable parameter: one thread per parameter, sum over the batch
__global__ void grad_kernel(const float* X, const float* H1, const float* H2, const float* dZ1,
                            const float* dZ2, const float* dout, int64_t B, float* G) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NW) return;
    const int q = p + OFF_W1;
    float s = 0.f;
    if (q < OFF_B1) {  // W1[j][k]
        const int j = (q - OFF_W1) / NF, k = (q - OFF_W1) % NF;
        for (int64_t i = 0; i < B; ++i) s = fmaf(dZ1[i * NH + j], X[i * NF + k], s);
    } else if (q < OFF_W2) {  // b1[j]
        const int j = q - OFF_B1;
        for (int64_t i = 0; i < B; ++i) s += dZ1[i * NH + j];
    } else if (q < OFF_B2) {  // W2[j][k]
        const int j = (q - OFF_W2) / NH, k = (q - OFF_W2) % NH;
        for (int64_t i = 0; i < B; ++i) s = fmaf(dZ2[i * NH + j], H1[i * NH + k], s);
    } else if (q < OFF_W3) {  // b2[j]
        const int j = q - OFF_B2;
        for (int64_t i = 0; i < B; ++i) s += dZ2[i * NH + j];
    } else if (q < OFF_B3) {  // w3[k]
        const int k = q - OFF_W3;
        for (int64_t i = 0; i < B; ++i) s = fmaf(dout[i], H2[i * NH + k], s);
    } else {  // b3
        for (int64_t i = 0; i < B; ++i) s += dout[i];
    }
    G[p] = s;
}

__global__ void adam_kernel(float* P, const float* G, float* M, float* V, float lr, float b1,
                            float b2, float epsa, int step) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NW) return;
    const float g = G[p];
    const float m = b1 * M[p] + (1.f - b1) * g;
    const float v = b2 * V[p] + (1.f - b2) * g * g;
    M[p] = m;
    V[p] = v;
    const float mh = m / (1.f - powf(b1, (float)step)), vh = v / (1.f - powf(b2, (float)step));
    P[OFF_W1 + p] -= lr * mh / (sqrtf(vh) + epsa);
}

// counter-based hash (SplitMix64 finaliser) for the mini-batch draws
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__global__ void draw_kernel(uint64_t seed, int step, int64_t n, int64_t B, int64_t* idx) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < B) idx[i] = (int64_t)(mix64(seed ^ mix64(((uint64_t)step << 32) + (uint64_t)i)) % (uint64_t)n);
}

unsigned nb(int64_t n) { return (unsigned)hm_cdiv(n, 256); }

struct Scratch {
    std::vector<DevBuf> bufs;
    float* alloc(size_t n, cudaStream_t st) { return (float*)hm_dmalloc(bufs, n * 4, st, true); }
    ~Scratch() {
        for (DevBuf& d : bufs) cudaFree(d.p);
    }
};

// forward pass of the standardised batch X (B x 6): Z1, H1, Z2, H2, out
void forward(const float* dP, const float* X, int64_t B, float* Z1, float* H1, float* Z2,
             float* H2, float* out, const float* Y, float* dout, cudaStream_t st) {
    dense_fwd_kernel<<<nb(B * NH), 256, 0, st>>>(X, NF, dP + OFF_W1, dP + OFF_B1, NH, B, Z1, H1);
    HM_LAUNCHED();
    dense_fwd_kernel<<<nb(B * NH), 256, 0, st>>>(H1, NH, dP + OFF_W2, dP + OFF_B2, NH, B, Z2, H2);
    HM_LAUNCHED();
    head_kernel<<<nb(B), 256, 0, st>>>(H2, dP, Y, B, out, dout);
    HM_LAUNCHED();
    HM_CUDA(cudaGetLastError());
}

}  // namespace

// Predictions (standardised target units) of a model for raw features, all on the device.
void rank_model_predict_dev(const float* dP, const float* dF, int64_t n, float* dOut,
                            cudaStream_t st) {
    if (n <= 0) return;
    Scratch S;
    float* X = S.alloc(n * NF, st);
    float* Z1 = S.alloc(n * NH, st);
    float* H1 = S.alloc(n * NH, st);
    float* Z2 = S.alloc(n * NH, st);
    float* H2 = S.alloc(n * NH, st);
    gather_std_kernel<<<nb(n), 256, 0, st>>>(dF, nullptr, dP, nullptr, n, X, nullptr);
    HM_LAUNCHED();
    forward(dP, X, n, Z1, H1, Z2, H2, dOut, nullptr, nullptr, st);
    HM_CUDA(cudaStreamSynchronize(st));
}

extern "C" {

hm_status hm_rank_model_predict(const float* params, const float* feats, int64_t n, float* out,
                                void* stream) {
    try {
        if (n < 0 || (n > 0 && (!params || !feats || !out))) hm_throw(HM_ERR_ARG, "null pointer");
        rank_model_predict_dev(params, feats, n, out, (cudaStream_t)stream);
    } catch (const hm_error& e) {
        hm_set_error(e.msg);
        return e.st;
    } catch (...) {
        hm_set_error("unexpected internal error");
        return HM_ERR_CUDA;
    }
    return HM_OK;
}

hm_status hm_rank_model_train(const float* feats, const float* targets, int64_t n, int32_t steps,
                              int32_t batch, float lr, uint64_t seed, float* params,
                              float* loss, void* stream) {
    try {
        if (!feats || !targets || !params || n < 2 || steps < 0 || batch < 1 || !(lr > 0))
            hm_throw(HM_ERR_ARG, "invalid training arguments");
        cudaStream_t st = (cudaStream_t)stream;
        // standardisation constants on the host (the data set is small)
        std::vector<float> hF((size_t)n * NF), hT(n), hP(NPARAM, 0.f);
        HM_CUDA(cudaMemcpyAsync(hF.data(), feats, hF.size() * 4, cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaMemcpyAsync(hT.data(), targets, hT.size() * 4, cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaMemcpyAsync(hP.data(), params, NPARAM * 4, cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaStreamSynchronize(st));
        for (int f = 0; f < NF + 1; ++f) {
            double s = 0, s2 = 0;
            for (int64_t i = 0; i < n; ++i) {
                const double v = f < NF ? hF[i * NF + f] : hT[i];
                s += v;
                s2 += v * v;
            }
            const double mu = s / n, sd = std::sqrt(std::max(s2 / n - mu * mu, 1e-12));
            if (f < NF) {
                hP[f] = (float)mu;
                hP[NF + f] = (float)sd;
            } else {
                hP[12] = (float)mu;
                hP[13] = (float)sd;
            }
        }
        HM_CUDA(cudaMemcpyAsync(params, hP.data(), 14 * 4, cudaMemcpyHostToDevice, st));
        const int64_t B = std::min<int64_t>(batch, n);
        Scratch S;
        int64_t* idx = (int64_t*)hm_dmalloc(S.bufs, B * 8, st, false);
        float* X = S.alloc(B * NF, st);
        float* Y = S.alloc(B, st);
        float* Z1 = S.alloc(B * NH, st);
        float* H1 = S.alloc(B * NH, st);
        float* Z2 = S.alloc(B * NH, st);
        float* H2 = S.alloc(B * NH, st);
        float* out = S.alloc(B, st);
        float* dout = S.alloc(B, st);
        float* dZ2 = S.alloc(B * NH, st);
        float* dZ1 = S.alloc(B * NH, st);
        float* G = S.alloc(NW, st);
        float* M = S.alloc(NW, st);
        float* V = S.alloc(NW, st);
        std::vector<float> hout(B), hy(B);
        for (int step = 1; step <= steps; ++step) {
            draw_kernel<<<nb(B), 256, 0, st>>>(seed, step, n, B, idx);
            HM_LAUNCHED();
            gather_std_kernel<<<nb(B), 256, 0, st>>>(feats, targets, params, idx, B, X, Y);
            HM_LAUNCHED();
            forward(params, X, B, Z1, H1, Z2, H2, out, Y, dout, st);
            back_head_kernel<<<nb(B * NH), 256, 0, st>>>(dout, params, Z2, B, dZ2);
            HM_LAUNCHED();
            back_hidden_kernel<<<nb(B * NH), 256, 0, st>>>(dZ2, params, Z1, B, dZ1);
            HM_LAUNCHED();
            grad_kernel<<<nb(NW), 256, 0, st>>>(X, H1, H2, dZ1, dZ2, dout, B, G);
            HM_LAUNCHED();
            adam_kernel<<<nb(NW), 256, 0, st>>>(params, G, M, V, lr, 0.9f, 0.999f, 1e-8f, step);
            HM_LAUNCHED();
            HM_CUDA(cudaGetLastError());
            if (loss) {  // mean squared error of this step's batch (standardised units)
                HM_CUDA(cudaMemcpyAsync(hout.data(), out, B * 4, cudaMemcpyDeviceToHost, st));
                HM_CUDA(cudaMemcpyAsync(hy.data(), Y, B * 4, cudaMemcpyDeviceToHost, st));
                HM_CUDA(cudaStreamSynchronize(st));
                double e = 0;
                for (int64_t i = 0; i < B; ++i) e += (double)(hout[i] - hy[i]) * (hout[i] - hy[i]);
                loss[step - 1] = (float)(e / B);
            }
        }
        HM_CUDA(cudaStreamSynchronize(st));
    } catch (const hm_error& e) {
        hm_set_error(e.msg);
        return e.st;
    } catch (...) {
        hm_set_error("unexpected internal error");
        return HM_ERR_CUDA;
    }
    return HM_OK;
}

hm_status hm_rank_model_grad(const float* params, const float* feats, const float* targets,
                             int64_t n, float* grad, float* loss, void* stream) {
    // full-batch loss and gradient of the trainable parameters (for checks)
    try {
        if (!params || !feats || !targets || !grad || n < 1) hm_throw(HM_ERR_ARG, "null pointer");
        cudaStream_t st = (cudaStream_t)stream;
        Scratch S;
        float* X = S.alloc(n * NF, st);
        float* Y = S.alloc(n, st);
        float* Z1 = S.alloc(n * NH, st);
        float* H1 = S.alloc(n * NH, st);
        float* Z2 = S.alloc(n * NH, st);
        float* H2 = S.alloc(n * NH, st);
        float* out = S.alloc(n, st);
        float* dout = S.alloc(n, st);
        float* dZ2 = S.alloc(n * NH, st);
        float* dZ1 = S.alloc(n * NH, st);
        gather_std_kernel<<<nb(n), 256, 0, st>>>(feats, targets, params, nullptr, n, X, Y);
        HM_LAUNCHED();
        forward(params, X, n, Z1, H1, Z2, H2, out, Y, dout, st);
        back_head_kernel<<<nb(n * NH), 256, 0, st>>>(dout, params, Z2, n, dZ2);
        HM_LAUNCHED();
        back_hidden_kernel<<<nb(n * NH), 256, 0, st>>>(dZ2, params, Z1, n, dZ1);
        HM_LAUNCHED();
        grad_kernel<<<nb(NW), 256, 0, st>>>(X, H1, H2, dZ1, dZ2, dout, n, grad);
        HM_LAUNCHED();
        HM_CUDA(cudaGetLastError());
        if (loss) {
            std::vector<float> ho(n), hy(n);
            HM_CUDA(cudaMemcpyAsync(ho.data(), out, n * 4, cudaMemcpyDeviceToHost, st));
            HM_CUDA(cudaMemcpyAsync(hy.data(), Y, n * 4, cudaMemcpyDeviceToHost, st));
            HM_CUDA(cudaStreamSynchronize(st));
            double e = 0;
            for (int64_t i = 0; i < n; ++i) e += (double)(ho[i] - hy[i]) * (ho[i] - hy[i]);
            *loss = (float)(e / n);
        }
        HM_CUDA(cudaStreamSynchronize(st));
    } catch (const hm_error& e) {
        hm_set_error(e.msg);
        return e.st;
    } catch (...) {
        hm_set_error("unexpected internal error");
        return HM_ERR_CUDA;
    }
    return HM_OK;
}

}  // extern "C"
