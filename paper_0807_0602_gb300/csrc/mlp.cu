// Surrogate network of include/mlp.h: 6 -> 128 -> 128 -> 128 -> 3 with the
// exact GELU, bfloat16 GEMM operands and FP32 accumulation on the tensor
// cores (mma.sync.m16n8k16), FP32 biases, activations and Adam state.
//
// The GEMMs here are tiny (at most 128 x 128 weights against a batch of a
// few thousand rows), so every kernel works on 16-row batch tiles with one
// CTA of four warps; fragments are assembled element by element from shared
// or global memory.  Weight gradients are reduced over the batch inside one
// CTA per output block, in a fixed order, so training is deterministic.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "mlp.h"

namespace {

constexpr int NL = 4;
// valid fan-in / fan-out per layer, and both padded to the mma tile (16, 8)
__host__ __device__ constexpr int IN(int l) { return l == 0 ? 6 : 128; }
__host__ __device__ constexpr int OUT(int l) { return l == 3 ? 3 : 128; }
__host__ __device__ constexpr int KP(int l) { return l == 0 ? 16 : 128; }
__host__ __device__ constexpr int NP(int l) { return l == 3 ? 8 : 128; }

struct Dev {
    float* theta;          // FP32 master parameters, flat layer order
    float* m;              // Adam first moment
    float* v;              // Adam second moment
    float* grad;           // gradient scratch [MLP_N_PARAMS]
    __nv_bfloat16* Wp[NL]; // padded bfloat16 weights [KP][NP]
    int woff[NL], boff[NL];
    // activation scratch for max_batch rows
    __nv_bfloat16* A[NL];  // layer inputs (bf16) [rows][KP]
    float* Z[NL - 1];      // hidden pre-activations [rows][128]
    float* DZ[NL];         // dL/dz per layer [rows][NP]
    float* Y;              // outputs [rows][3]
    float* lpart;          // per-tile partial losses
};

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[16 x 8] += A[16 x K] B[K x 8] with element accessors A(m, k), B(k, n).
// Fragment layout of m16n8k16: lane = 4 g + q; A holds rows g, g + 8 and
// columns 2q, 2q + 1, 2q + 8, 2q + 9; B holds rows 2q, 2q + 1, 2q + 8,
// 2q + 9 of column g; C holds (g, 2q), (g, 2q + 1), (g + 8, 2q), (g + 8, 2q + 1).
template <class FA, class FB>
__device__ __forceinline__ void tile_mma(float (&c)[4], FA A, FB B, int K) {
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t a[4], b[2];
        a[0] = pack2(A(g, k0 + 2 * q), A(g, k0 + 2 * q + 1));
        a[1] = pack2(A(g + 8, k0 + 2 * q), A(g + 8, k0 + 2 * q + 1));
        a[2] = pack2(A(g, k0 + 2 * q + 8), A(g, k0 + 2 * q + 9));
        a[3] = pack2(A(g + 8, k0 + 2 * q + 8), A(g + 8, k0 + 2 * q + 9));
        b[0] = pack2(B(k0 + 2 * q, g), B(k0 + 2 * q + 1, g));
        b[1] = pack2(B(k0 + 2 * q + 8, g), B(k0 + 2 * q + 9, g));
        mma16816(c, a, b);
    }
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// Forward pass of one 16-row tile; TRAIN keeps the layer inputs and
// pre-activations for the backward pass.
template <bool TRAIN>
__global__ void __launch_bounds__(128) k_fwd(Dev d, const float* __restrict__ X, int n, float* __restrict__ Y) {
    __shared__ __nv_bfloat16 act[2][16][128 + 8];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, q = lane & 3;
    const int row0 = blockIdx.x * 16;
    for (int i = tid; i < 16 * 16; i += 128) {
        const int r = i >> 4, c = i & 15;
        const float v = (row0 + r < n && c < 6) ? X[(long long)(row0 + r) * 6 + c] : 0.0f;
        const __nv_bfloat16 b = __float2bfloat16_rn(v);
        act[0][r][c] = b;
        if (TRAIN && row0 + r < n) d.A[0][(long long)(row0 + r) * 16 + c] = b;
    }
    __syncthreads();
    for (int l = 0; l < NL; ++l) {
        const int cur = l & 1, nxt = cur ^ 1;
        const int N = NP(l), K = KP(l);
        const __nv_bfloat16* W = d.Wp[l];
        const float* bias = d.theta + d.boff[l];
        for (int nt = warp; nt < N / 8; nt += 4) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            tile_mma(
                c, [&](int m, int k) { return act[cur][m][k]; },
                [&](int k, int nn) { return W[k * N + nt * 8 + nn]; }, K);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int r = g + (e >> 1) * 8, col = nt * 8 + 2 * q + (e & 1);
                const bool row_ok = row0 + r < n;
                if (l < NL - 1) {
                    const float z = c[e] + bias[col];
                    const __nv_bfloat16 h = __float2bfloat16_rn(gelu(z));
                    act[nxt][r][col] = h;
                    if (TRAIN && row_ok) {
                        d.Z[l][(long long)(row0 + r) * 128 + col] = z;
                        d.A[l + 1][(long long)(row0 + r) * 128 + col] = h;
                    }
                } else if (col < 3 && row_ok) {
                    Y[(long long)(row0 + r) * 3 + col] = c[e] + bias[col];
                }
            }
        }
        __syncthreads();
    }
}

// Backward through the activations of one 16-row tile: dL/dz for every layer
// (FP32), and the tile's partial sum of squared errors.
__global__ void __launch_bounds__(128) k_bwd(Dev d, const float* __restrict__ T, int n) {
    __shared__ __nv_bfloat16 dzb[16][128 + 8];
    __shared__ float sq[16 * 3];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, q = lane & 3;
    const int row0 = blockIdx.x * 16;
    const float scale = 2.0f / (float)(n * 3);
    for (int i = tid; i < 16 * 16; i += 128) {
        const int r = i >> 4, c = i & 15;
        float dz = 0.0f;
        if (row0 + r < n && c < 3) {
            const float e = d.Y[(long long)(row0 + r) * 3 + c] - T[(long long)(row0 + r) * 3 + c];
            dz = scale * e;
            sq[r * 3 + c] = e * e;
        } else if (c < 3) {
            sq[r * 3 + c] = 0.0f;
        }
        if (row0 + r < n && c < 8) d.DZ[3][(long long)(row0 + r) * 8 + c] = dz;
        dzb[r][c] = __float2bfloat16_rn(dz);
    }
    __syncthreads();
    if (tid == 0) {
        float s = 0.0f;
        for (int i = 0; i < 48; ++i) s += sq[i];
        d.lpart[blockIdx.x] = s;
    }
    for (int l = NL - 1; l >= 1; --l) {
        // dh = dz_l W_l^T  (K = padded fan-out of layer l, N = 128 inputs of layer l)
        const int Kd = l == NL - 1 ? 16 : 128;
        const int NPl = NP(l), Nv = OUT(l);
        const __nv_bfloat16* W = d.Wp[l];
        float acc[4][4];
        for (int j = 0; j < 4; ++j) {
            const int nt = warp + 4 * j;
            acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
            tile_mma(
                acc[j], [&](int m, int k) { return dzb[m][k]; },
                [&](int k, int nn) {
                    return k < Nv ? W[(nt * 8 + nn) * NPl + k] : __float2bfloat16_rn(0.0f);
                },
                Kd);
        }
        __syncthreads();   // every warp has read dzb
        for (int j = 0; j < 4; ++j) {
            const int nt = warp + 4 * j;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int r = g + (e >> 1) * 8, col = nt * 8 + 2 * q + (e & 1);
                float dz = 0.0f;
                if (row0 + r < n) {
                    dz = acc[j][e] * gelu_grad(d.Z[l - 1][(long long)(row0 + r) * 128 + col]);
                    d.DZ[l - 1][(long long)(row0 + r) * 128 + col] = dz;
                }
                dzb[r][col] = __float2bfloat16_rn(dz);
            }
        }
        __syncthreads();
    }
}

// Weight gradient of one 16 x 32 block (in x out) of layer l:
// gW = A_l^T bf16(DZ_l), summed over the batch rows in order.
struct WBlock {
    int l, m0, n0;
};

__global__ void __launch_bounds__(128) k_wgrad(Dev d, const WBlock* __restrict__ blocks, int n) {
    const WBlock wb = blocks[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const int l = wb.l;
    const int nt0 = wb.n0 + warp * 8;
    if (nt0 >= NP(l)) return;
    const int lda = KP(l), ldz = NP(l);
    const __nv_bfloat16* A = d.A[l];
    const float* DZ = d.DZ[l];
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    const int Kr = (n + 15) / 16 * 16;
    tile_mma(
        c,
        [&](int m, int k) { return k < n ? A[(long long)k * lda + wb.m0 + m] : __float2bfloat16_rn(0.0f); },
        [&](int k, int nn) { return __float2bfloat16_rn(k < n ? DZ[(long long)k * ldz + nt0 + nn] : 0.0f); }, Kr);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int m = wb.m0 + g + (e >> 1) * 8, col = nt0 + 2 * q + (e & 1);
        if (m < IN(l) && col < OUT(l)) d.grad[d.woff[l] + m * OUT(l) + col] = c[e];
    }
}

// Bias gradients: one thread per output unit sums dz over the rows in order.
__global__ void k_bgrad(Dev d, int n) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    for (int l = 0; l < NL; ++l) {
        if (j < OUT(l)) {
            float s = 0.0f;
            for (int r = 0; r < n; ++r) s += d.DZ[l][(long long)r * NP(l) + j];
            d.grad[d.boff[l] + j] = s;
            return;
        }
        j -= OUT(l);
    }
}

__global__ void k_loss(const float* __restrict__ part, int ntiles, int n, float* __restrict__ out) {
    float s = 0.0f;
    for (int i = 0; i < ntiles; ++i) s += part[i];
    *out = s / (float)(n * 3);
}

__global__ void k_adam(Dev d, const float* __restrict__ g, int N, float lr, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float m = 0.9f * d.m[i] + 0.1f * gi;
        const float v = 0.999f * d.v[i] + 0.001f * gi * gi;
        d.m[i] = m;
        d.v[i] = v;
        d.theta[i] -= lr * (m * c1) / (sqrtf(v * c2) + 1e-8f);
    }
}

// Refreshes the padded bfloat16 weights from the FP32 master copy.
__global__ void k_pack(Dev d) {
    for (int l = 0; l < NL; ++l) {
        const int tot = KP(l) * NP(l);
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += gridDim.x * blockDim.x) {
            const int k = i / NP(l), c = i - k * NP(l);
            const float w = (k < IN(l) && c < OUT(l)) ? d.theta[d.woff[l] + k * OUT(l) + c] : 0.0f;
            d.Wp[l][i] = __float2bfloat16_rn(w);
        }
    }
}

}  // namespace

struct mlp_s {
    Dev d;
    int max_batch = 0;
    int64_t steps = 0;
    cudaStream_t stream = nullptr;
    std::vector<void*> allocs;
    WBlock* d_blocks = nullptr;
    int nblocks = 0;
    float* d_loss = nullptr;
};

namespace {

int fail(cudaError_t e) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? MLP_ENOMEM : MLP_ECUDA;
}

template <typename T>
T* mal(mlp_t* h, size_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, count * sizeof(T) + 16) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    h->allocs.push_back(p);
    return static_cast<T*>(p);
}

int forward_impl(mlp_t* h, const float* x, int n, float* y, bool train) {
    const int tiles = (n + 15) / 16;
    if (train) k_fwd<true><<<tiles, 128, 0, h->stream>>>(h->d, x, n, y);
    else k_fwd<false><<<tiles, 128, 0, h->stream>>>(h->d, x, n, y);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MLP_OK : fail(e);
}

int grad_impl(mlp_t* h, const float* x, const float* t, int n, float* loss) {
    int rc = forward_impl(h, x, n, h->d.Y, true);
    if (rc) return rc;
    const int tiles = (n + 15) / 16;
    k_bwd<<<tiles, 128, 0, h->stream>>>(h->d, t, n);
    k_wgrad<<<h->nblocks, 128, 0, h->stream>>>(h->d, h->d_blocks, n);
    k_bgrad<<<(128 * 3 + 3 + 127) / 128, 128, 0, h->stream>>>(h->d, n);
    k_loss<<<1, 1, 0, h->stream>>>(h->d.lpart, tiles, n, loss ? loss : h->d_loss);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MLP_OK : fail(e);
}

}  // namespace

extern "C" {

int mlp_create(int max_batch, const float* params, void* stream, mlp_t** out) {
    if (!out || max_batch < 1 || max_batch > (1 << 24)) return MLP_EINVAL;
    *out = nullptr;
    mlp_t* h = new mlp_s();
    h->max_batch = max_batch;
    h->stream = static_cast<cudaStream_t>(stream);
    Dev& d = h->d;
    int o = 0;
    for (int l = 0; l < NL; ++l) {
        d.woff[l] = o;
        o += IN(l) * OUT(l);
        d.boff[l] = o;
        o += OUT(l);
    }
    const size_t rows = (size_t)(max_batch + 15) / 16 * 16;
    d.theta = mal<float>(h, MLP_N_PARAMS);
    d.m = mal<float>(h, MLP_N_PARAMS);
    d.v = mal<float>(h, MLP_N_PARAMS);
    d.grad = mal<float>(h, MLP_N_PARAMS);
    for (int l = 0; l < NL; ++l) {
        d.Wp[l] = mal<__nv_bfloat16>(h, (size_t)KP(l) * NP(l));
        d.A[l] = mal<__nv_bfloat16>(h, rows * KP(l));
        d.DZ[l] = mal<float>(h, rows * NP(l));
    }
    for (int l = 0; l < NL - 1; ++l) d.Z[l] = mal<float>(h, rows * 128);
    d.Y = mal<float>(h, rows * 3);
    d.lpart = mal<float>(h, rows / 16 + 1);
    h->d_loss = mal<float>(h, 1);
    std::vector<WBlock> blocks;
    for (int l = 0; l < NL; ++l)
        for (int m0 = 0; m0 < KP(l); m0 += 16)
            for (int n0 = 0; n0 < NP(l); n0 += 32) blocks.push_back({l, m0, n0});
    h->nblocks = (int)blocks.size();
    h->d_blocks = mal<WBlock>(h, blocks.size());
    for (void* p : h->allocs)
        if (!p) {
            mlp_destroy(h);
            return MLP_ENOMEM;
        }
    bool ok = d.theta && d.m && d.v && d.grad && d.Y && d.lpart && h->d_loss && h->d_blocks;
    for (int l = 0; l < NL; ++l) ok = ok && d.Wp[l] && d.A[l] && d.DZ[l];
    for (int l = 0; l < NL - 1; ++l) ok = ok && d.Z[l];
    if (!ok) {
        mlp_destroy(h);
        return MLP_ENOMEM;
    }
    if (cudaMemcpy(h->d_blocks, blocks.data(), blocks.size() * sizeof(WBlock), cudaMemcpyHostToDevice) != cudaSuccess) {
        mlp_destroy(h);
        return MLP_ECUDA;
    }
    std::vector<float> init(MLP_N_PARAMS, 0.0f);
    if (params) memcpy(init.data(), params, sizeof(float) * MLP_N_PARAMS);
    int rc = mlp_set_params(h, init.data());
    if (rc) {
        mlp_destroy(h);
        return rc;
    }
    *out = h;
    return MLP_OK;
}

int mlp_set_params(mlp_t* h, const float* params) {
    if (!h || !params) return MLP_EINVAL;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) e = cudaMemcpy(h->d.theta, params, sizeof(float) * MLP_N_PARAMS, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(h->d.m, 0, sizeof(float) * MLP_N_PARAMS);
    if (e == cudaSuccess) e = cudaMemset(h->d.v, 0, sizeof(float) * MLP_N_PARAMS);
    if (e != cudaSuccess) return fail(e);
    k_pack<<<64, 256, 0, h->stream>>>(h->d);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(e);
    h->steps = 0;
    return MLP_OK;
}

int mlp_get_params(mlp_t* h, float* params) {
    if (!h || !params) return MLP_EINVAL;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) e = cudaMemcpy(params, h->d.theta, sizeof(float) * MLP_N_PARAMS, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? MLP_OK : fail(e);
}

int mlp_forward(mlp_t* h, const float* x, int n, float* y) {
    if (!h || !x || !y || n < 1 || n > h->max_batch) return MLP_EINVAL;
    return forward_impl(h, x, n, y, false);
}

int mlp_gradients(mlp_t* h, const float* x, const float* t, int n, float* grad, float* loss) {
    if (!h || !x || !t || !grad || n < 1 || n > h->max_batch) return MLP_EINVAL;
    int rc = grad_impl(h, x, t, n, loss);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(grad, h->d.grad, sizeof(float) * MLP_N_PARAMS, cudaMemcpyDeviceToDevice, h->stream);
    return e == cudaSuccess ? MLP_OK : fail(e);
}

int mlp_train_step(mlp_t* h, const float* x, const float* t, int n, float lr, float* loss) {
    if (!h || !x || !t || n < 1 || n > h->max_batch || !std::isfinite(lr)) return MLP_EINVAL;
    int rc = grad_impl(h, x, t, n, loss);
    if (rc) return rc;
    h->steps += 1;
    const double c1 = 1.0 / (1.0 - std::pow(0.9, (double)h->steps));
    const double c2 = 1.0 / (1.0 - std::pow(0.999, (double)h->steps));
    k_adam<<<64, 256, 0, h->stream>>>(h->d, h->d.grad, MLP_N_PARAMS, lr, (float)c1, (float)c2);
    k_pack<<<64, 256, 0, h->stream>>>(h->d);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MLP_OK : fail(e);
}

int64_t mlp_step_count(const mlp_t* h) { return h ? h->steps : -1; }

void mlp_destroy(mlp_t* h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    for (void* p : h->allocs)
        if (p) cudaFree(p);
    cudaGetLastError();
    delete h;
}

}  // extern "C"
