// lbm_mlp.cu -- the surrogate network of the hybrid method: an ensemble of
// multilayer perceptrons mapping a throat's geometry (three radii, three centre
// distances, contact angle) to its entry pressure and sampled p_c - S_w curve,
// trained and evaluated entirely by the kernels below.
//
// Every layer is a GEMM on the tensor cores (mma.sync m16n8k16, BF16 or FP16
// operands rounded from FP32 master values while the tiles are staged in shared
// memory, FP32 accumulation) with the bias, ReLU or ReLU-derivative mask fused
// into the epilogue.  Operands are described by strides, so the forward pass
// (H W^T), the input gradient (dZ W) and the weight gradient (dZ^T H) share one
// kernel.  Mean squared error, bias gradients and Adam are elementwise kernels.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm_internal.h"

namespace lbmk {

namespace {

constexpr int BM = 64, BN = 64, BK = 32, GEMM_THREADS = 128, KPAD = 8;
constexpr float LOSS_SCALE = 1024.f;

enum Epi : int { EPI_NONE = 0, EPI_BIAS = 1, EPI_BIAS_RELU = 2, EPI_MASK = 3 };

template <class T>
struct Op;
template <>
struct Op<__nv_bfloat16> {
    static __device__ __forceinline__ __nv_bfloat16 cvt(float v) { return __float2bfloat16_rn(v); }
    static __device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
};
template <>
struct Op<__half> {
    static __device__ __forceinline__ __half cvt(float v) { return __float2half_rn(v); }
    static __device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
};

struct GemmArgs {
    const float* A;  // A(m, k) = A[m * sam + k * sak]
    const float* B;  // B(k, n) = B[k * sbk + n * sbn]
    float* C;        // C[m * ldc + n]
    int M, N, K;
    int sam, sak, sbk, sbn, ldc;
    const float* bias;  // per n (EPI_BIAS*)
    const float* mask;  // mask[m * ldm + n] > 0 keeps the value (EPI_MASK)
    int ldm;
    int epi;
};

// C = A B with the epilogue; 64 x 64 tile per CTA, four warps of 32 x 32.
template <class T>
__global__ void __launch_bounds__(GEMM_THREADS) gemm_kernel(GemmArgs p) {
    __shared__ __align__(16) T As[BM][BK + KPAD];
    __shared__ __align__(16) T Bs[BN][BK + KPAD];  // Bs[n][k]
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int wm = warp >> 1, wn = warp & 1;
    const int gid = lane >> 2, tig = lane & 3;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

    for (int k0 = 0; k0 < p.K; k0 += BK) {
#pragma unroll
        for (int r = 0; r < (BM * BK) / GEMM_THREADS; ++r) {
            const int i = tid + r * GEMM_THREADS;
            const int m = i / BK, k = i % BK;
            const int gm = m0 + m, gk = k0 + k;
            const float v = (gm < p.M && gk < p.K) ? p.A[(size_t)gm * p.sam + (size_t)gk * p.sak] : 0.f;
            As[m][k] = Op<T>::cvt(v);
        }
#pragma unroll
        for (int r = 0; r < (BN * BK) / GEMM_THREADS; ++r) {
            const int i = tid + r * GEMM_THREADS;
            const int n = i / BK, k = i % BK;
            const int gn = n0 + n, gk = k0 + k;
            const float v = (gn < p.N && gk < p.K) ? p.B[(size_t)gk * p.sbk + (size_t)gn * p.sbn] : 0.f;
            Bs[n][k] = Op<T>::cvt(v);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r0 = wm * 32 + i * 16 + gid;
                a[i][0] = *reinterpret_cast<const uint32_t*>(&As[r0][kk + tig * 2]);
                a[i][1] = *reinterpret_cast<const uint32_t*>(&As[r0 + 8][kk + tig * 2]);
                a[i][2] = *reinterpret_cast<const uint32_t*>(&As[r0][kk + 8 + tig * 2]);
                a[i][3] = *reinterpret_cast<const uint32_t*>(&As[r0 + 8][kk + 8 + tig * 2]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c0 = wn * 32 + j * 8 + gid;
                b[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[c0][kk + tig * 2]);
                b[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[c0][kk + 8 + tig * 2]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) Op<T>::mma(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int m = m0 + wm * 32 + i * 16 + gid + (r >= 2 ? 8 : 0);
                const int n = n0 + wn * 32 + j * 8 + tig * 2 + (r & 1);
                if (m >= p.M || n >= p.N) continue;
                float v = acc[i][j][r];
                if (p.epi == EPI_BIAS || p.epi == EPI_BIAS_RELU) v += p.bias[n];
                if (p.epi == EPI_BIAS_RELU) v = fmaxf(v, 0.f);
                if (p.epi == EPI_MASK && !(p.mask[(size_t)m * p.ldm + n] > 0.f)) v = 0.f;
                p.C[(size_t)m * p.ldc + n] = v;
            }
}

// dY = loss_scale * 2 (Y - T) / (rows * cols); loss partial sums per block.
// The backward GEMMs round their operands to 16 bits: the loss scale keeps the
// small backpropagated values clear of FP16's subnormal range; gradients are
// divided by it again before they are used.
__global__ void mse_grad_kernel(const float* __restrict__ Y, const float* __restrict__ T, float* __restrict__ dY,
                                int count, float scale, float loss_scale, double* __restrict__ loss_sum) {
    __shared__ double red[8];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const float d = Y[i] - T[i];
        dY[i] = 2.f * d * scale * loss_scale;
        acc += (double)d * (double)d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        atomicAdd(loss_sum, s * (double)scale);
    }
}

// db[o] = sum_b dZ[b * out + o]
__global__ void bias_grad_kernel(const float* __restrict__ dZ, float* __restrict__ db, int rows, int out) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= out) return;
    float s = 0.f;
    for (int b = 0; b < rows; ++b) s += dZ[(size_t)b * out + o];
    db[o] = s;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1,
                            float c2, float inv_scale) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i] * inv_scale;
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void gather_rows_kernel(const float* __restrict__ src, const int* __restrict__ idx, float* __restrict__ dst,
                                   int rows, int cols) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows * cols; i += gridDim.x * blockDim.x) {
        const int r = i / cols, c = i % cols;
        dst[i] = src[(size_t)idx[r] * cols + c];
    }
}

// Per output: mean and standard deviation over the ensemble members.
__global__ void ensemble_stats_kernel(const float* __restrict__ Ys, int members, int count, float* __restrict__ mean,
                                      float* __restrict__ spread) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int m = 0; m < members; ++m) s += Ys[(size_t)m * count + i];
        const float mu = s / members;
        float q = 0.f;
        for (int m = 0; m < members; ++m) {
            const float d = Ys[(size_t)m * count + i] - mu;
            q += d * d;
        }
        mean[i] = mu;
        spread[i] = members > 1 ? sqrtf(q / (members - 1)) : 0.f;
    }
}

// splitmix64 and Box-Muller for the seeded He-normal initialisation (host)
uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double uniform01(uint64_t& s) { return ((splitmix(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

}  // namespace

}  // namespace lbmk

using namespace lbmk;

struct lbm_surrogate {
    lbm_surrogate_config cfg;
    std::vector<int> sizes;     // n_in, hidden..., n_out
    std::vector<size_t> w_off;  // offsets of W_l and b_l in a member's flat parameter block
    std::vector<size_t> b_off;
    size_t n_params;
    float* params;  // [members][n_params]
    float* grads;   // [n_params] (one member at a time)
    float* adam_m;  // [members][n_params]
    float* adam_v;
    int adam_t[64];
    float* acts;    // activations for a batch: layer inputs + output
    float* dbuf[2];  // gradient ping-pong buffers
    int cap_rows;    // rows the activation buffers hold
    double* d_loss;
    cudaStream_t stream;
};

namespace {

int sur_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

#define SUR_CUDA(call)                                    \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return sur_fail(e_, #call); \
    } while (0)

size_t act_width(const lbm_surrogate* s) {
    size_t w = 0;
    for (int x : s->sizes) w = std::max(w, (size_t)x);
    return w;
}

// activation buffer of layer input l (l = 0: network input, L: output)
float* act(lbm_surrogate* s, int l) { return s->acts + (size_t)l * s->cap_rows * act_width(s); }

int ensure_rows(lbm_surrogate* s, int rows) {
    if (rows <= s->cap_rows) return LBM_OK;
    cudaFree(s->acts);
    cudaFree(s->dbuf[0]);
    cudaFree(s->dbuf[1]);
    s->acts = s->dbuf[0] = s->dbuf[1] = nullptr;
    s->cap_rows = 0;
    const size_t w = act_width(s);
    SUR_CUDA(cudaMalloc(&s->acts, sizeof(float) * s->sizes.size() * rows * w));
    SUR_CUDA(cudaMalloc(&s->dbuf[0], sizeof(float) * rows * w));
    SUR_CUDA(cudaMalloc(&s->dbuf[1], sizeof(float) * rows * w));
    s->cap_rows = rows;
    return LBM_OK;
}

cudaError_t gemm(const lbm_surrogate* s, const GemmArgs& a) {
    dim3 grid((a.N + BN - 1) / BN, (a.M + BM - 1) / BM);
    if (s->cfg.half) gemm_kernel<__half><<<grid, GEMM_THREADS, 0, s->stream>>>(a);
    else gemm_kernel<__nv_bfloat16><<<grid, GEMM_THREADS, 0, s->stream>>>(a);
    return cudaGetLastError();
}

// forward of member m on rows already in act(s, 0)
int forward(lbm_surrogate* s, int m, int rows) {
    const float* P = s->params + (size_t)m * s->n_params;
    const int L = (int)s->sizes.size() - 1;
    for (int l = 0; l < L; ++l) {
        GemmArgs a{};
        a.A = act(s, l);
        a.sam = s->sizes[l];
        a.sak = 1;
        a.B = P + s->w_off[l];  // B(k, n) = W[n][k]
        a.sbk = 1;
        a.sbn = s->sizes[l];
        a.C = act(s, l + 1);
        a.ldc = s->sizes[l + 1];
        a.M = rows;
        a.N = s->sizes[l + 1];
        a.K = s->sizes[l];
        a.bias = P + s->b_off[l];
        a.epi = l < L - 1 ? EPI_BIAS_RELU : EPI_BIAS;
        SUR_CUDA(gemm(s, a));
    }
    return LBM_OK;
}

// gradients of the MSE of member m on rows (targets T on the device) into
// s->grads; the batch loss is added to *loss_acc (device)
int backward(lbm_surrogate* s, int m, int rows, const float* T, double* loss_acc) {
    const float* P = s->params + (size_t)m * s->n_params;
    const int L = (int)s->sizes.size() - 1;
    const int nout = s->sizes[L];
    float* dz = s->dbuf[0];
    float* dh = s->dbuf[1];
    const int count = rows * nout;
    mse_grad_kernel<<<std::min(1024, (count + 255) / 256), 256, 0, s->stream>>>(act(s, L), T, dz, count,
                                                                                  1.0f / (float)count, LOSS_SCALE,
                                                                                  loss_acc);
    SUR_CUDA(cudaGetLastError());
    for (int l = L - 1; l >= 0; --l) {
        const int in = s->sizes[l], out = s->sizes[l + 1];
        GemmArgs g{};  // dW = dZ^T H : (out x in), K = rows
        g.A = dz;
        g.sam = 1;
        g.sak = out;
        g.B = act(s, l);
        g.sbk = in;
        g.sbn = 1;
        g.C = s->grads + s->w_off[l];
        g.ldc = in;
        g.M = out;
        g.N = in;
        g.K = rows;
        g.epi = EPI_NONE;
        SUR_CUDA(gemm(s, g));
        bias_grad_kernel<<<(out + 127) / 128, 128, 0, s->stream>>>(dz, s->grads + s->b_off[l], rows, out);
        SUR_CUDA(cudaGetLastError());
        if (l > 0) {
            GemmArgs d{};  // dH = dZ W, masked by ReLU'(z_{l-1}) = [h_l > 0]
            d.A = dz;
            d.sam = out;
            d.sak = 1;
            d.B = P + s->w_off[l];
            d.sbk = in;
            d.sbn = 1;
            d.C = dh;
            d.ldc = in;
            d.M = rows;
            d.N = in;
            d.K = out;
            d.mask = act(s, l);
            d.ldm = in;
            d.epi = EPI_MASK;
            SUR_CUDA(gemm(s, d));
            std::swap(dz, dh);
        }
    }
    return LBM_OK;
}

int adam(lbm_surrogate* s, int m, float lr) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const int t = ++s->adam_t[m];
    const float c1 = 1.f - std::pow(b1, (float)t), c2 = 1.f - std::pow(b2, (float)t);
    const int n = (int)s->n_params;
    adam_kernel<<<std::min(1024, (n + 255) / 256), 256, 0, s->stream>>>(
        s->params + (size_t)m * s->n_params, s->grads, s->adam_m + (size_t)m * s->n_params,
        s->adam_v + (size_t)m * s->n_params, n, lr, b1, b2, eps, c1, c2, 1.0f / LOSS_SCALE);
    SUR_CUDA(cudaGetLastError());
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_surrogate_create(const lbm_surrogate_config* cfg, void* stream, lbm_surrogate** out) {
    if (!cfg || !out || cfg->n_in < 1 || cfg->n_out < 1 || cfg->n_hidden < 1 || cfg->n_layers < 1 ||
        cfg->n_members < 1 || cfg->n_members > 64 || cfg->n_in > 4096 || cfg->n_hidden > 4096 || cfg->n_out > 4096 ||
        cfg->n_layers > 16) {
        set_error("lbm_surrogate_create: bad configuration");
        return LBM_ERR_ARG;
    }
    lbm_surrogate* s = new (std::nothrow) lbm_surrogate();
    if (!s) { set_error("host allocation failed"); return LBM_ERR_OOM; }
    s->cfg = *cfg;
    s->stream = (cudaStream_t)stream;
    s->sizes.push_back(cfg->n_in);
    for (int i = 0; i < cfg->n_layers; ++i) s->sizes.push_back(cfg->n_hidden);
    s->sizes.push_back(cfg->n_out);
    size_t off = 0;
    for (size_t l = 0; l + 1 < s->sizes.size(); ++l) {
        s->w_off.push_back(off);
        off += (size_t)s->sizes[l] * s->sizes[l + 1];
        s->b_off.push_back(off);
        off += (size_t)s->sizes[l + 1];
    }
    s->n_params = off;
    // seeded He-normal weights, zero biases, per member
    std::vector<float> init(s->n_params * cfg->n_members, 0.f);
    for (int m = 0; m < cfg->n_members; ++m) {
        uint64_t st = cfg->seed * 0x100000001B3ull + (uint64_t)m * 0x9E3779B97F4A7C15ull + 1;
        for (size_t l = 0; l + 1 < s->sizes.size(); ++l) {
            const double sd = std::sqrt(2.0 / s->sizes[l]);
            const size_t nw = (size_t)s->sizes[l] * s->sizes[l + 1];
            for (size_t i = 0; i < nw; ++i) {
                const double u1 = uniform01(st), u2 = uniform01(st);
                init[m * s->n_params + s->w_off[l] + i] =
                    (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
            }
        }
    }
    auto bail = [&](int rc) { lbm_surrogate_destroy(s); return rc; };
    const size_t pb = sizeof(float) * s->n_params * cfg->n_members;
    cudaError_t e;
    if ((e = cudaMalloc(&s->params, pb)) != cudaSuccess) return bail(sur_fail(e, "cudaMalloc"));
    if ((e = cudaMalloc(&s->adam_m, pb)) != cudaSuccess) return bail(sur_fail(e, "cudaMalloc"));
    if ((e = cudaMalloc(&s->adam_v, pb)) != cudaSuccess) return bail(sur_fail(e, "cudaMalloc"));
    if ((e = cudaMalloc(&s->grads, sizeof(float) * s->n_params)) != cudaSuccess) return bail(sur_fail(e, "cudaMalloc"));
    if ((e = cudaMalloc(&s->d_loss, sizeof(double))) != cudaSuccess) return bail(sur_fail(e, "cudaMalloc"));
    if ((e = cudaMemcpyAsync(s->params, init.data(), pb, cudaMemcpyHostToDevice, s->stream)) != cudaSuccess)
        return bail(sur_fail(e, "cudaMemcpyAsync"));
    if ((e = cudaMemsetAsync(s->adam_m, 0, pb, s->stream)) != cudaSuccess) return bail(sur_fail(e, "memset"));
    if ((e = cudaMemsetAsync(s->adam_v, 0, pb, s->stream)) != cudaSuccess) return bail(sur_fail(e, "memset"));
    if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return bail(sur_fail(e, "sync"));
    *out = s;
    return LBM_OK;
}

int lbm_surrogate_num_params(const lbm_surrogate* s) { return s ? (int)s->n_params : 0; }

int lbm_surrogate_get_params(lbm_surrogate* s, int member, float* out) {
    if (!s || !out || member < 0 || member >= s->cfg.n_members) { set_error("bad argument"); return LBM_ERR_ARG; }
    SUR_CUDA(cudaMemcpyAsync(out, s->params + (size_t)member * s->n_params, sizeof(float) * s->n_params,
                             cudaMemcpyDeviceToHost, s->stream));
    SUR_CUDA(cudaStreamSynchronize(s->stream));
    return LBM_OK;
}

int lbm_surrogate_set_params(lbm_surrogate* s, int member, const float* in) {
    if (!s || !in || member < 0 || member >= s->cfg.n_members) { set_error("bad argument"); return LBM_ERR_ARG; }
    SUR_CUDA(cudaMemcpyAsync(s->params + (size_t)member * s->n_params, in, sizeof(float) * s->n_params,
                             cudaMemcpyHostToDevice, s->stream));
    SUR_CUDA(cudaStreamSynchronize(s->stream));
    s->adam_t[member] = 0;
    SUR_CUDA(cudaMemsetAsync(s->adam_m + (size_t)member * s->n_params, 0, sizeof(float) * s->n_params, s->stream));
    SUR_CUDA(cudaMemsetAsync(s->adam_v + (size_t)member * s->n_params, 0, sizeof(float) * s->n_params, s->stream));
    return LBM_OK;
}

int lbm_surrogate_forward(lbm_surrogate* s, int member, const float* X, int n, float* Y) {
    if (!s || !X || !Y || n < 1 || member < 0 || member >= s->cfg.n_members) {
        set_error("bad argument");
        return LBM_ERR_ARG;
    }
    if (int rc = ensure_rows(s, n)) return rc;
    const int L = (int)s->sizes.size() - 1;
    SUR_CUDA(cudaMemcpyAsync(act(s, 0), X, sizeof(float) * n * s->cfg.n_in, cudaMemcpyHostToDevice, s->stream));
    if (int rc = forward(s, member, n)) return rc;
    SUR_CUDA(cudaMemcpyAsync(Y, act(s, L), sizeof(float) * n * s->cfg.n_out, cudaMemcpyDeviceToHost, s->stream));
    SUR_CUDA(cudaStreamSynchronize(s->stream));
    return LBM_OK;
}

int lbm_surrogate_gradients(lbm_surrogate* s, int member, const float* X, const float* T, int n, float* grads,
                            double* loss) {
    if (!s || !X || !T || !grads || n < 1 || member < 0 || member >= s->cfg.n_members) {
        set_error("bad argument");
        return LBM_ERR_ARG;
    }
    if (int rc = ensure_rows(s, n)) return rc;
    float* dT = nullptr;
    SUR_CUDA(cudaMallocAsync(&dT, sizeof(float) * n * s->cfg.n_out, s->stream));
    SUR_CUDA(cudaMemcpyAsync(act(s, 0), X, sizeof(float) * n * s->cfg.n_in, cudaMemcpyHostToDevice, s->stream));
    SUR_CUDA(cudaMemcpyAsync(dT, T, sizeof(float) * n * s->cfg.n_out, cudaMemcpyHostToDevice, s->stream));
    SUR_CUDA(cudaMemsetAsync(s->d_loss, 0, sizeof(double), s->stream));
    int rc = forward(s, member, n);
    if (!rc) rc = backward(s, member, n, dT, s->d_loss);
    cudaFreeAsync(dT, s->stream);
    if (rc) return rc;
    SUR_CUDA(cudaMemcpyAsync(grads, s->grads, sizeof(float) * s->n_params, cudaMemcpyDeviceToHost, s->stream));
    double l = 0;
    SUR_CUDA(cudaMemcpyAsync(&l, s->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    SUR_CUDA(cudaStreamSynchronize(s->stream));
    for (size_t i = 0; i < s->n_params; ++i) grads[i] /= LOSS_SCALE;
    if (loss) *loss = l;
    return LBM_OK;
}

int lbm_surrogate_train(lbm_surrogate* s, const float* X, const float* T, int n, int epochs, int batch, float lr,
                        unsigned long long shuffle_seed, double* epoch_loss) {
    if (!s || !X || !T || n < 1 || epochs < 0 || batch < 1 || !(lr > 0.f)) {
        set_error("lbm_surrogate_train: bad argument");
        return LBM_ERR_ARG;
    }
    const int nin = s->cfg.n_in, nout = s->cfg.n_out, L = (int)s->sizes.size() - 1;
    batch = std::min(batch, n);
    if (int rc = ensure_rows(s, batch)) return rc;
    float *dX = nullptr, *dT = nullptr, *dTb = nullptr;
    int* dIdx = nullptr;
    double* dLoss = nullptr;
    auto cleanup = [&]() {
        cudaFree(dX); cudaFree(dT); cudaFree(dTb); cudaFree(dIdx); cudaFree(dLoss);
    };
#define TR_CUDA(call)                               \
    do {                                            \
        cudaError_t e_ = (call);                    \
        if (e_ != cudaSuccess) {                    \
            cleanup();                              \
            return sur_fail(e_, #call);             \
        }                                           \
    } while (0)
    TR_CUDA(cudaMalloc(&dX, sizeof(float) * (size_t)n * nin));
    TR_CUDA(cudaMalloc(&dT, sizeof(float) * (size_t)n * nout));
    TR_CUDA(cudaMalloc(&dTb, sizeof(float) * (size_t)batch * nout));
    TR_CUDA(cudaMalloc(&dIdx, sizeof(int) * (size_t)n * std::max(1, epochs)));
    TR_CUDA(cudaMalloc(&dLoss, sizeof(double) * (size_t)s->cfg.n_members * std::max(1, epochs)));
    TR_CUDA(cudaMemcpyAsync(dX, X, sizeof(float) * (size_t)n * nin, cudaMemcpyHostToDevice, s->stream));
    TR_CUDA(cudaMemcpyAsync(dT, T, sizeof(float) * (size_t)n * nout, cudaMemcpyHostToDevice, s->stream));
    TR_CUDA(cudaMemsetAsync(dLoss, 0, sizeof(double) * (size_t)s->cfg.n_members * std::max(1, epochs), s->stream));
    for (int m = 0; m < s->cfg.n_members; ++m) {
        // seeded Fisher-Yates order per member and epoch
        std::vector<int> order((size_t)n * std::max(1, epochs));
        uint64_t st = shuffle_seed * 0x9E3779B97F4A7C15ull + (uint64_t)m * 0xD1B54A32D192ED03ull + 7;
        for (int ep = 0; ep < epochs; ++ep) {
            int* o = order.data() + (size_t)ep * n;
            for (int i = 0; i < n; ++i) o[i] = i;
            for (int i = n - 1; i > 0; --i) std::swap(o[i], o[splitmix(st) % (uint64_t)(i + 1)]);
        }
        TR_CUDA(cudaMemcpyAsync(dIdx, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice, s->stream));
        TR_CUDA(cudaStreamSynchronize(s->stream));  // the host order buffer is reused
        for (int ep = 0; ep < epochs; ++ep) {
            for (int b0 = 0; b0 + batch <= n; b0 += batch) {
                const int* idx = dIdx + (size_t)ep * n + b0;
                gather_rows_kernel<<<std::min(1024, (batch * nin + 255) / 256), 256, 0, s->stream>>>(dX, idx, act(s, 0),
                                                                                                 batch, nin);
                gather_rows_kernel<<<std::min(1024, (batch * nout + 255) / 256), 256, 0, s->stream>>>(dT, idx, dTb,
                                                                                                  batch, nout);
                int rc = forward(s, m, batch);
                if (!rc) rc = backward(s, m, batch, dTb, dLoss + (size_t)m * epochs + ep);
                if (!rc) rc = adam(s, m, lr);
                if (rc) {
                    cleanup();
                    return rc;
                }
            }
        }
    }
    if (epoch_loss && epochs > 0) {
        TR_CUDA(cudaMemcpyAsync(epoch_loss, dLoss, sizeof(double) * (size_t)s->cfg.n_members * epochs,
                                cudaMemcpyDeviceToHost, s->stream));
    }
    TR_CUDA(cudaStreamSynchronize(s->stream));
    // per-epoch loss = mean over batches of the batch MSE
    if (epoch_loss) {
        const int nb = n / batch;
        for (int i = 0; i < s->cfg.n_members * epochs; ++i) epoch_loss[i] /= std::max(1, nb);
    }
    cleanup();
#undef TR_CUDA
    (void)L;
    return LBM_OK;
}

int lbm_surrogate_predict(lbm_surrogate* s, const float* X, int n, float* mean, float* spread) {
    if (!s || !X || !mean || !spread || n < 1) {
        set_error("lbm_surrogate_predict: bad argument");
        return LBM_ERR_ARG;
    }
    const int nin = s->cfg.n_in, nout = s->cfg.n_out, M = s->cfg.n_members, L = (int)s->sizes.size() - 1;
    const int chunk = std::min(n, 16384);
    if (int rc = ensure_rows(s, chunk)) return rc;
    float *dYs = nullptr, *dMean = nullptr, *dSpread = nullptr;
    auto cleanup = [&]() { cudaFree(dYs); cudaFree(dMean); cudaFree(dSpread); };
    cudaError_t e;
    if ((e = cudaMalloc(&dYs, sizeof(float) * (size_t)M * chunk * nout)) != cudaSuccess) { cleanup(); return sur_fail(e, "cudaMalloc"); }
    if ((e = cudaMalloc(&dMean, sizeof(float) * (size_t)chunk * nout)) != cudaSuccess) { cleanup(); return sur_fail(e, "cudaMalloc"); }
    if ((e = cudaMalloc(&dSpread, sizeof(float) * (size_t)chunk * nout)) != cudaSuccess) { cleanup(); return sur_fail(e, "cudaMalloc"); }
    for (int r0 = 0; r0 < n; r0 += chunk) {
        const int rows = std::min(chunk, n - r0);
        if ((e = cudaMemcpyAsync(act(s, 0), X + (size_t)r0 * nin, sizeof(float) * rows * nin, cudaMemcpyHostToDevice,
                                 s->stream)) != cudaSuccess) { cleanup(); return sur_fail(e, "cudaMemcpyAsync"); }
        for (int m = 0; m < M; ++m) {
            if (int rc = forward(s, m, rows)) { cleanup(); return rc; }
            if ((e = cudaMemcpyAsync(dYs + (size_t)m * rows * nout, act(s, L), sizeof(float) * rows * nout,
                                     cudaMemcpyDeviceToDevice, s->stream)) != cudaSuccess) { cleanup(); return sur_fail(e, "copy"); }
        }
        ensemble_stats_kernel<<<std::min(1024, (rows * nout + 255) / 256), 256, 0, s->stream>>>(dYs, M, rows * nout,
                                                                                               dMean, dSpread);
        if ((e = cudaGetLastError()) != cudaSuccess) { cleanup(); return sur_fail(e, "ensemble_stats_kernel"); }
        if ((e = cudaMemcpyAsync(mean + (size_t)r0 * nout, dMean, sizeof(float) * rows * nout, cudaMemcpyDeviceToHost,
                                 s->stream)) != cudaSuccess) { cleanup(); return sur_fail(e, "copy"); }
        if ((e = cudaMemcpyAsync(spread + (size_t)r0 * nout, dSpread, sizeof(float) * rows * nout,
                                 cudaMemcpyDeviceToHost, s->stream)) != cudaSuccess) { cleanup(); return sur_fail(e, "copy"); }
        if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) { cleanup(); return sur_fail(e, "sync"); }
    }
    cleanup();
    return LBM_OK;
}

void lbm_surrogate_destroy(lbm_surrogate* s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    cudaFree(s->params);
    cudaFree(s->grads);
    cudaFree(s->adam_m);
    cudaFree(s->adam_v);
    cudaFree(s->acts);
    cudaFree(s->dbuf[0]);
    cudaFree(s->dbuf[1]);
    cudaFree(s->d_loss);
    delete s;
}

}  // extern "C"
