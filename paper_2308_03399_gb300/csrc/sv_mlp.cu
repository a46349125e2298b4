// Learned cost model: a small MLP (n_in -> H -> H -> 1, ReLU) that predicts
// the log run time of a circuit under a candidate configuration, trained on
// timings the simulator itself produces.  Forward pass, backward pass (mean
// squared error) and the Adam update are hand-written kernels; nothing here
// uses a library GEMM.
//
// Parameter layout (one float32 array):
//   W1 [H x n_in] | b1 [H] | W2 [H x H] | b2 [H] | w3 [H] | b3 [1]
//
// Determinism: every sample's forward/backward runs in one thread, and the
// per-parameter gradient is summed over samples in index order by one
// thread, so results do not depend on launch order.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sv.h"

namespace sv {
void set_last_error(const std::string& msg);  // sv_runtime.cu
}

struct sv_mlp_s {
    int n_in = 0, H = 0;
    size_t n_par = 0;
    float* par = nullptr;   // device parameters
    float* m = nullptr;     // Adam first moment
    float* v = nullptr;     // Adam second moment
    float* grad = nullptr;  // summed gradient
    // per-batch work buffers (grown on demand)
    int cap = 0;
    float *x = nullptr, *t = nullptr, *h1 = nullptr, *h2 = nullptr, *y = nullptr, *gs = nullptr, *loss = nullptr;
    int64_t step = 0;
    cudaStream_t stream = nullptr;
};

namespace {

constexpr int MLP_MAX_IN = 64;
constexpr int MLP_MAX_H = 128;

__host__ __device__ inline size_t n_params(int n_in, int H) { return (size_t)H * n_in + H + (size_t)H * H + H + H + 1; }

// one thread per sample: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = w3.h2 + b3
__global__ void k_mlp_forward(const float* __restrict__ par, int n_in, int H, const float* __restrict__ x, int N,
                              float* __restrict__ h1, float* __restrict__ h2, float* __restrict__ y) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const float* W1 = par;
    const float* b1 = W1 + (size_t)H * n_in;
    const float* W2 = b1 + H;
    const float* b2 = W2 + (size_t)H * H;
    const float* w3 = b2 + H;
    const float* b3 = w3 + H;
    const float* xs = x + (size_t)s * n_in;
    float* a1 = h1 + (size_t)s * H;
    float* a2 = h2 + (size_t)s * H;
    for (int j = 0; j < H; ++j) {
        float z = b1[j];
        for (int i = 0; i < n_in; ++i) z += W1[(size_t)j * n_in + i] * xs[i];
        a1[j] = z > 0.f ? z : 0.f;
    }
    for (int j = 0; j < H; ++j) {
        float z = b2[j];
        for (int i = 0; i < H; ++i) z += W2[(size_t)j * H + i] * a1[i];
        a2[j] = z > 0.f ? z : 0.f;
    }
    float out = b3[0];
    for (int i = 0; i < H; ++i) out += w3[i] * a2[i];
    y[s] = out;
}

// one thread per sample: gradient of 0.5 * (y - t)^2 / N with respect to
// every parameter, written to that sample's row of gs [N x n_par]
__global__ void k_mlp_backward(const float* __restrict__ par, int n_in, int H, const float* __restrict__ x,
                               const float* __restrict__ t, int N, const float* __restrict__ h1,
                               const float* __restrict__ h2, const float* __restrict__ y, float* __restrict__ gs,
                               float* __restrict__ loss) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const size_t P = n_params(n_in, H);
    const float* W2 = par + (size_t)H * n_in + H;
    const float* w3 = W2 + (size_t)H * H + H;
    const float* xs = x + (size_t)s * n_in;
    const float* a1 = h1 + (size_t)s * H;
    const float* a2 = h2 + (size_t)s * H;
    float* g = gs + (size_t)s * P;
    float* gW1 = g;
    float* gb1 = gW1 + (size_t)H * n_in;
    float* gW2 = gb1 + H;
    float* gb2 = gW2 + (size_t)H * H;
    float* gw3 = gb2 + H;
    float* gb3 = gw3 + H;
    const float e = y[s] - t[s];
    loss[s] = 0.5f * e * e / N;
    const float dy = e / N;
    float d2[MLP_MAX_H], d1[MLP_MAX_H];
    for (int j = 0; j < H; ++j) {
        gw3[j] = dy * a2[j];
        d2[j] = a2[j] > 0.f ? dy * w3[j] : 0.f;  // through relu
    }
    gb3[0] = dy;
    for (int j = 0; j < H; ++j) {
        gb2[j] = d2[j];
        for (int i = 0; i < H; ++i) gW2[(size_t)j * H + i] = d2[j] * a1[i];
    }
    for (int i = 0; i < H; ++i) {
        float z = 0.f;
        for (int j = 0; j < H; ++j) z += W2[(size_t)j * H + i] * d2[j];
        d1[i] = a1[i] > 0.f ? z : 0.f;
    }
    for (int j = 0; j < H; ++j) {
        gb1[j] = d1[j];
        for (int i = 0; i < n_in; ++i) gW1[(size_t)j * n_in + i] = d1[j] * xs[i];
    }
}

// one thread per parameter: sum over samples in index order
__global__ void k_mlp_sum(const float* __restrict__ gs, int N, size_t P, float* __restrict__ grad,
                          const float* __restrict__ loss, float* __restrict__ loss_out) {
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P) {
        float s = 0.f;
        for (int n = 0; n < N; ++n) s += gs[(size_t)n * P + p];
        grad[p] = s;
    }
    if (p == 0 && loss_out) {
        float l = 0.f;
        for (int n = 0; n < N; ++n) l += loss[n];
        *loss_out = l;
    }
}

// Adam (Kingma and Ba, 2015)
__global__ void k_mlp_adam(float* __restrict__ par, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ grad, size_t P, float lr, float b1, float b2, float eps,
                           float c1, float c2) {
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const float g = grad[p];
    const float mp = b1 * m[p] + (1.f - b1) * g;
    const float vp = b2 * v[p] + (1.f - b2) * g * g;
    m[p] = mp;
    v[p] = vp;
    par[p] -= lr * (mp / c1) / (sqrtf(vp / c2) + eps);
}

sv_status mfail(sv_status s, const char* msg) {
    sv::set_last_error(msg);
    return s;
}

sv_status ensure_cap(sv_mlp m, int N) {
    if (N <= m->cap) return SV_OK;
    cudaFree(m->x);
    cudaFree(m->t);
    cudaFree(m->h1);
    cudaFree(m->h2);
    cudaFree(m->y);
    cudaFree(m->gs);
    cudaFree(m->loss);
    m->x = m->t = m->h1 = m->h2 = m->y = m->gs = m->loss = nullptr;
    const size_t P = m->n_par;
    if (cudaMalloc(&m->x, sizeof(float) * (size_t)N * m->n_in) != cudaSuccess ||
        cudaMalloc(&m->t, sizeof(float) * N) != cudaSuccess ||
        cudaMalloc(&m->h1, sizeof(float) * (size_t)N * m->H) != cudaSuccess ||
        cudaMalloc(&m->h2, sizeof(float) * (size_t)N * m->H) != cudaSuccess ||
        cudaMalloc(&m->y, sizeof(float) * N) != cudaSuccess ||
        cudaMalloc(&m->gs, sizeof(float) * (size_t)N * P) != cudaSuccess ||
        cudaMalloc(&m->loss, sizeof(float) * (N + 1)) != cudaSuccess) {
        cudaGetLastError();
        m->cap = 0;
        return mfail(SV_ENOMEM, "sv_mlp: cannot allocate work buffers");
    }
    m->cap = N;
    return SV_OK;
}

sv_status forward(sv_mlp m, int N) {
    k_mlp_forward<<<(N + 127) / 128, 128, 0, m->stream>>>(m->par, m->n_in, m->H, m->x, N, m->h1, m->h2, m->y);
    return cudaGetLastError() == cudaSuccess ? SV_OK : mfail(SV_ECUDA, "sv_mlp: forward launch failed");
}

sv_status backward(sv_mlp m, int N) {
    k_mlp_backward<<<(N + 127) / 128, 128, 0, m->stream>>>(m->par, m->n_in, m->H, m->x, m->t, N, m->h1, m->h2, m->y,
                                                           m->gs, m->loss);
    const size_t P = m->n_par;
    k_mlp_sum<<<(unsigned)((P + 255) / 256), 256, 0, m->stream>>>(m->gs, N, P, m->grad, m->loss, m->loss + N);
    return cudaGetLastError() == cudaSuccess ? SV_OK : mfail(SV_ECUDA, "sv_mlp: backward launch failed");
}

}  // namespace

extern "C" {

sv_status sv_mlp_create(int n_in, int n_hidden, sv_mlp* out) {
    if (!out) return mfail(SV_EINVAL, "sv_mlp_create: out is NULL");
    *out = nullptr;
    if (n_in < 1 || n_in > MLP_MAX_IN || n_hidden < 1 || n_hidden > MLP_MAX_H)
        return mfail(SV_EINVAL, "sv_mlp_create: n_in must be 1..64 and n_hidden 1..128");
    sv_mlp m = new sv_mlp_s();
    m->n_in = n_in;
    m->H = n_hidden;
    m->n_par = n_params(n_in, n_hidden);
    if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&m->par, sizeof(float) * m->n_par) != cudaSuccess ||
        cudaMalloc(&m->m, sizeof(float) * m->n_par) != cudaSuccess ||
        cudaMalloc(&m->v, sizeof(float) * m->n_par) != cudaSuccess ||
        cudaMalloc(&m->grad, sizeof(float) * m->n_par) != cudaSuccess) {
        cudaGetLastError();
        sv_mlp_free(m);
        return mfail(SV_ENOMEM, "sv_mlp_create: cannot allocate parameters");
    }
    cudaMemsetAsync(m->par, 0, sizeof(float) * m->n_par, m->stream);
    cudaMemsetAsync(m->m, 0, sizeof(float) * m->n_par, m->stream);
    cudaMemsetAsync(m->v, 0, sizeof(float) * m->n_par, m->stream);
    *out = m;
    return SV_OK;
}

sv_status sv_mlp_free(sv_mlp m) {
    if (!m) return SV_OK;
    if (m->stream) cudaStreamSynchronize(m->stream);
    cudaFree(m->par);
    cudaFree(m->m);
    cudaFree(m->v);
    cudaFree(m->grad);
    cudaFree(m->x);
    cudaFree(m->t);
    cudaFree(m->h1);
    cudaFree(m->h2);
    cudaFree(m->y);
    cudaFree(m->gs);
    cudaFree(m->loss);
    if (m->stream) cudaStreamDestroy(m->stream);
    delete m;
    return SV_OK;
}

uint64_t sv_mlp_num_params(sv_mlp m) { return m ? (uint64_t)m->n_par : 0; }

sv_status sv_mlp_set_params(sv_mlp m, const float* params, uint64_t n) {
    if (!m || !params || n != m->n_par) return mfail(SV_EINVAL, "sv_mlp_set_params: bad arguments");
    if (cudaMemcpyAsync(m->par, params, sizeof(float) * n, cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->m, 0, sizeof(float) * n, m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->v, 0, sizeof(float) * n, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
        return mfail(SV_ECUDA, "sv_mlp_set_params: copy failed");
    m->step = 0;
    return SV_OK;
}

sv_status sv_mlp_get_params(sv_mlp m, float* params, uint64_t n) {
    if (!m || !params || n != m->n_par) return mfail(SV_EINVAL, "sv_mlp_get_params: bad arguments");
    if (cudaMemcpyAsync(params, m->par, sizeof(float) * n, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
        return mfail(SV_ECUDA, "sv_mlp_get_params: copy failed");
    return SV_OK;
}

sv_status sv_mlp_forward(sv_mlp m, const float* x, int n, float* y) {
    if (!m || !x || !y || n < 1) return mfail(SV_EINVAL, "sv_mlp_forward: bad arguments");
    sv_status st = ensure_cap(m, n);
    if (st) return st;
    cudaMemcpyAsync(m->x, x, sizeof(float) * (size_t)n * m->n_in, cudaMemcpyHostToDevice, m->stream);
    if ((st = forward(m, n))) return st;
    if (cudaMemcpyAsync(y, m->y, sizeof(float) * n, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
        return mfail(SV_ECUDA, "sv_mlp_forward: failed");
    return SV_OK;
}

sv_status sv_mlp_gradient(sv_mlp m, const float* x, const float* t, int n, float* loss, float* grad) {
    if (!m || !x || !t || n < 1) return mfail(SV_EINVAL, "sv_mlp_gradient: bad arguments");
    sv_status st = ensure_cap(m, n);
    if (st) return st;
    cudaMemcpyAsync(m->x, x, sizeof(float) * (size_t)n * m->n_in, cudaMemcpyHostToDevice, m->stream);
    cudaMemcpyAsync(m->t, t, sizeof(float) * n, cudaMemcpyHostToDevice, m->stream);
    if ((st = forward(m, n)) || (st = backward(m, n))) return st;
    if (grad) cudaMemcpyAsync(grad, m->grad, sizeof(float) * m->n_par, cudaMemcpyDeviceToHost, m->stream);
    if (loss) cudaMemcpyAsync(loss, m->loss + n, sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) return mfail(SV_ECUDA, "sv_mlp_gradient: failed");
    return SV_OK;
}

sv_status sv_mlp_train(sv_mlp m, const float* x, const float* t, int n, int epochs, int batch, float lr,
                       uint64_t seed, float* final_loss) {
    if (!m || !x || !t || n < 1 || epochs < 1 || batch < 1) return mfail(SV_EINVAL, "sv_mlp_train: bad arguments");
    if (batch > n) batch = n;
    sv_status st = ensure_cap(m, n);
    if (st) return st;
    // shuffled minibatches: the host permutes sample order every epoch
    // (splitmix64 keyed by seed and epoch) and uploads each minibatch
    std::vector<int> order(n);
    std::vector<float> xb((size_t)batch * m->n_in), tb(batch);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int e = 0; e < epochs; ++e) {
        for (int i = 0; i < n; ++i) order[i] = i;
        uint64_t z = seed * 0x9E3779B97F4A7C15ull + (uint64_t)e;
        for (int i = n - 1; i > 0; --i) {
            z += 0x9E3779B97F4A7C15ull;
            uint64_t r = z;
            r = (r ^ (r >> 30)) * 0xBF58476D1CE4E5B9ull;
            r = (r ^ (r >> 27)) * 0x94D049BB133111EBull;
            r ^= r >> 31;
            const int j = (int)(r % (uint64_t)(i + 1));
            const int tmp = order[i];
            order[i] = order[j];
            order[j] = tmp;
        }
        for (int b0 = 0; b0 + batch <= n; b0 += batch) {
            for (int k = 0; k < batch; ++k) {
                memcpy(&xb[(size_t)k * m->n_in], x + (size_t)order[b0 + k] * m->n_in, sizeof(float) * m->n_in);
                tb[k] = t[order[b0 + k]];
            }
            cudaMemcpyAsync(m->x, xb.data(), sizeof(float) * xb.size(), cudaMemcpyHostToDevice, m->stream);
            cudaMemcpyAsync(m->t, tb.data(), sizeof(float) * batch, cudaMemcpyHostToDevice, m->stream);
            if ((st = forward(m, batch)) || (st = backward(m, batch))) break;
            m->step += 1;
            const float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
            k_mlp_adam<<<(unsigned)((m->n_par + 255) / 256), 256, 0, m->stream>>>(m->par, m->m, m->v, m->grad,
                                                                                 m->n_par, lr, b1, b2, eps, c1, c2);
            // the staging vectors are reused next minibatch: wait for the copies
            if (cudaStreamSynchronize(m->stream) != cudaSuccess) {
                st = mfail(SV_ECUDA, "sv_mlp_train: step failed");
                break;
            }
        }
        if (st) break;
    }
    if (st) return st;
    if (final_loss) {
        // mean squared error / 2 of the whole training set, final parameters
        std::vector<float> y(n);
        if ((st = sv_mlp_forward(m, x, n, y.data()))) return st;
        double l = 0.0;
        for (int i = 0; i < n; ++i) l += 0.5 * (double)(y[i] - t[i]) * (y[i] - t[i]);
        *final_loss = (float)(l / n);
    }
    return st;
}

}  // extern "C"
