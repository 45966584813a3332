// lbm_mlp.cu -- the surrogate network of the hybrid method: an ensemble of
// multilayer perceptrons mapping a throat's geometry (three radii, three centre
// distances, contact angle) to its entry pressure and sampled p_c - S_w curve,
// trained and evaluated entirely by the kernels below.
//
// Every layer is a GEMM on the fifth-generation tensor cores: one thread per CTA
// issues tcgen05.mma (BF16 or FP16 operands rounded from FP32 master values while
// the tiles are staged in shared memory, FP32 accumulation in tensor memory), and
// the four warps read the accumulator back with tcgen05.ld for the epilogue, which
// adds the bias, applies ReLU or the ReLU-derivative mask and writes rows through
// shared memory.  Operands are described by strides, so the forward pass (H W^T),
// the input gradient (dZ W) and the weight gradient (dZ^T H) share one kernel, and
// a third grid dimension runs all ensemble members of a layer in one launch.
// Mean squared error, bias gradients, Adam and the ensemble statistics are
// elementwise kernels.
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

// A CTA computes a TM x TN tile of C in chunks of TK along K, two chunks in flight.
constexpr int TM = 128, TN = 64, TK = 64, GEMM_THREADS = 128;
constexpr int A_TILE = TM * TK * 2, B_TILE = TN * TK * 2;  // bytes, 16-bit operands
constexpr int STAGE = A_TILE + B_TILE;
constexpr int GEMM_SMEM = 2 * STAGE + 64;  // two stages, then the barriers and the TMEM address
constexpr int EPI_LD = 33;                 // padded row of the epilogue's transpose buffer
constexpr float LOSS_SCALE = 1024.f;
constexpr unsigned long long GEMM_WAIT_NS = 2000000000ull;

enum Epi : int { EPI_NONE = 0, EPI_BIAS = 1, EPI_BIAS_RELU = 2, EPI_MASK = 3 };

template <class T>
struct Cvt;
template <>
struct Cvt<__nv_bfloat16> {
    static constexpr uint32_t kFormat = 1;  // instruction-descriptor operand format: BF16
    static __device__ __forceinline__ __nv_bfloat16 from(float v) { return __float2bfloat16_rn(v); }
};
template <>
struct Cvt<__half> {
    static constexpr uint32_t kFormat = 0;  // FP16
    static __device__ __forceinline__ __half from(float v) { return __float2half_rn(v); }
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
    // per ensemble member (grid z): element offsets of A, B, C, bias, mask
    long long zA, zB, zC, zBias, zMask;
    int* err;                    // set to 1 when a wait for the tensor cores ran out
    unsigned long long wait_ns;  // limit of each such wait
    int skip_mma;                // self-test only: issue no MMA, so that the waits run out
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Offset in bytes of element (r, k) of a K-major operand tile of TK columns in the
// tensor cores' interleaved layout without swizzle: 8 x 16-byte core matrices, the
// core matrices of one 8-row group adjacent along K (128 B apart), row groups
// TK / 8 core matrices (1024 B) apart.
__device__ __forceinline__ int core_offset(int r, int k) {
    return ((r >> 3) * (TK / 8) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}
constexpr uint32_t CORE_LBO = 128, CORE_SBO = (TK / 8) * 128;

// shared-memory matrix descriptor: start, leading and stride byte offsets (>> 4),
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((CORE_LBO >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((CORE_SBO >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of the given parity to complete, at most limit_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, unsigned long long limit_ns) {
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (true) {
        for (int i = 0; i < 64; ++i)
            if (mbar_test(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// Stage rows [r0, r0 + R) x columns [k0, k0 + TK) of X(r, k) = X[r * sr + k * sk]
// (zero outside rows x K) as 16-bit values into a core-matrix tile.  Consecutive
// threads walk whichever index is contiguous in memory; each thread issues eight
// loads before it converts and stores any of them.
template <class T, int R>
__device__ __forceinline__ void stage_tile(unsigned char* __restrict__ dst, const float* __restrict__ X, int sr,
                                           int sk, int r0, int rows, int k0, int K, int tid) {
    constexpr int PER = R * TK / GEMM_THREADS;
    static_assert(PER % 8 == 0, "tile elements per thread");
    const bool k_fast = sk == 1;
#pragma unroll 1
    for (int j0 = 0; j0 < PER; j0 += 8) {
        float v[8];
        int off[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int i = tid + (j0 + j) * GEMM_THREADS;
            const int r = k_fast ? i / TK : i % R, k = k_fast ? i % TK : i / R;
            const int gr = r0 + r, gk = k0 + k;
            off[j] = core_offset(r, k);
            v[j] = (gr < rows && gk < K) ? __ldg(X + (size_t)gr * sr + (size_t)gk * sk) : 0.f;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) *reinterpret_cast<T*>(dst + off[j]) = Cvt<T>::from(v[j]);
    }
}

#define TMEM_LD32(taddr, r)                                                                                       \
    asm volatile(                                                                                                 \
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18," \
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"                                         \
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),       \
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), \
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),            \
          "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),            \
          "=r"(r[30]), "=r"(r[31])                                                                              \
        : "r"(taddr))

// C = A B with the epilogue for ensemble member blockIdx.z.  The accumulator of the
// 128 x 64 tile lives in 64 columns of tensor memory (row m in lane m); thread 0
// issues the MMAs of a chunk while all threads stage the next one.
template <class T>
__global__ void __launch_bounds__(GEMM_THREADS) gemm_kernel(GemmArgs p) {
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * STAGE);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 2 * STAGE + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const long long z = blockIdx.z;
    const float* A = p.A + z * p.zA;
    const float* B = p.B + z * p.zB;
    float* C = p.C + z * p.zC;
    const uint32_t bar0 = smem_u32(&bars[0]), bar1 = smem_u32(&bars[1]);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                     "r"(TN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    // kind::f16 instruction descriptor: F32 accumulator, both operands K-major, N >> 3, M >> 4
    const uint32_t idesc = (1u << 4) | (Cvt<T>::kFormat << 7) | (Cvt<T>::kFormat << 10) |
                           ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

    const int nk = (p.K + TK - 1) / TK;
    int issued = 0;  // chunks whose MMAs were issued; the same in every thread
    bool failed = false;
    for (int c = 0; c < nk; ++c) {
        const int b = c & 1;
        unsigned char* sa = smem + b * STAGE;
        unsigned char* sb = sa + A_TILE;
        if (c >= 2) {  // chunk c - 2 used this stage: its MMAs must have finished reading it
            const bool ok = mbar_wait_bounded(b ? bar1 : bar0, (uint32_t)(((c - 2) >> 1) & 1), p.wait_ns);
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        }
        stage_tile<T, TM>(sa, A, p.sam, p.sak, m0, p.M, c * TK, p.K, tid);
        stage_tile<T, TN>(sb, B, p.sbn, p.sbk, n0, p.N, c * TK, p.K, tid);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (tid == 0 && !p.skip_mma) {
            const uint32_t a_addr = smem_u32(sa), b_addr = smem_u32(sb);
#pragma unroll
            for (int kk = 0; kk < TK / 16; ++kk) {  // K = 16 per MMA: two core matrices along K
                const uint64_t ad = smem_desc(a_addr + kk * 2 * 128);
                const uint64_t bd = smem_desc(b_addr + kk * 2 * 128);
                const uint32_t accumulate = (c > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             b ? bar1 : bar0)
                         : "memory");
        }
        issued = c + 1;
    }
    // The commit of the last chunk issued covers every MMA before it.
    const int last = issued - 1;
    const uint32_t last_bar = (last & 1) ? bar1 : bar0, last_parity = (uint32_t)((last >> 1) & 1);
    if (!failed && issued > 0) failed = __syncthreads_or(!mbar_wait_bounded(last_bar, last_parity, p.wait_ns));
    if (failed) {
        if (tid == 0) atomicOr(p.err, 1);
        // give the MMAs already issued a second bounded wait before their accumulator is freed
        if (issued > 0) mbar_wait_bounded(last_bar, last_parity, p.wait_ns);
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        if (warp == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TN) : "memory");
        return;
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

    // Epilogue: warp w owns rows 32 w .. 32 w + 31 (tensor-memory lanes); 32 columns
    // at a time go through a padded shared buffer so that a warp stores whole rows.
    float* buf = reinterpret_cast<float*>(smem) + warp * 32 * EPI_LD;
    const float* bias = p.bias ? p.bias + z * p.zBias : nullptr;
    const float* mask = p.mask ? p.mask + z * p.zMask : nullptr;
#pragma unroll 1
    for (int c0 = 0; c0 < TN && n0 + c0 < p.N; c0 += 32) {
        uint32_t r[32];
        TMEM_LD32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
        for (int j = 0; j < 32; ++j) buf[lane * EPI_LD + j] = __uint_as_float(r[j]);
        __syncwarp();
        const int n = n0 + c0 + lane;
        const float bn = (n < p.N && (p.epi == EPI_BIAS || p.epi == EPI_BIAS_RELU)) ? bias[n] : 0.f;
#pragma unroll 4
        for (int rr = 0; rr < 32; ++rr) {
            const int m = m0 + warp * 32 + rr;
            if (m >= p.M || n >= p.N) continue;
            float v = buf[rr * EPI_LD + lane] + bn;
            if (p.epi == EPI_BIAS_RELU) v = fmaxf(v, 0.f);
            if (p.epi == EPI_MASK && !(mask[(size_t)m * p.ldm + n] > 0.f)) v = 0.f;
            C[(size_t)m * p.ldc + n] = v;
        }
        __syncwarp();
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TN) : "memory");
}

// dY = loss_scale * 2 (Y - T) / (rows * cols); loss partial sums per block, for
// ensemble member blockIdx.y (member strides zY, zT, zL).
// The backward GEMMs round their operands to 16 bits: the loss scale keeps the
// small backpropagated values clear of FP16's subnormal range; gradients are
// divided by it again before they are used.
__global__ void mse_grad_kernel(const float* __restrict__ Y, const float* __restrict__ T, float* __restrict__ dY,
                                int count, float scale, float loss_scale, double* __restrict__ loss_sum,
                                long long zY, long long zT, long long zL) {
    __shared__ double red[8];
    const long long z = blockIdx.y;
    Y += z * zY;
    dY += z * zY;
    T += z * zT;
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
        atomicAdd(loss_sum + z * zL, s * (double)scale);
    }
}

// db[o] = sum_b dZ[b * out + o], member blockIdx.y
__global__ void bias_grad_kernel(const float* __restrict__ dZ, float* __restrict__ db, int rows, int out,
                                 long long zZ, long long zB) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= out) return;
    dZ += blockIdx.y * zZ;
    float s = 0.f;
    for (int b = 0; b < rows; ++b) s += dZ[(size_t)b * out + o];
    db[blockIdx.y * zB + o] = s;
}

// Bias corrections 1 - beta^t of each member (members keep their own step counts).
struct AdamCorrections {
    float c1[64], c2[64];
};

// Adam on the flat parameters of member blockIdx.y (n per member, contiguous)
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, AdamCorrections cc,
                            float inv_scale) {
    const size_t off = (size_t)blockIdx.y * n;
    const float c1 = cc.c1[blockIdx.y], c2 = cc.c2[blockIdx.y];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const size_t j = off + i;
        const float gi = g[j] * inv_scale;
        const float mi = b1 * m[j] + (1.f - b1) * gi;
        const float vi = b2 * v[j] + (1.f - b2) * gi * gi;
        m[j] = mi;
        v[j] = vi;
        p[j] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// dst (member blockIdx.y, rows x cols) = src rows idx[r]; member strides zIdx, zDst
__global__ void gather_rows_kernel(const float* __restrict__ src, const int* __restrict__ idx, float* __restrict__ dst,
                                   int rows, int cols, long long zIdx, long long zDst) {
    idx += blockIdx.y * zIdx;
    dst += blockIdx.y * zDst;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows * cols; i += gridDim.x * blockDim.x) {
        const int r = i / cols, c = i % cols;
        dst[i] = src[(size_t)idx[r] * cols + c];
    }
}

// Per output: mean and standard deviation over the ensemble members (member stride zY).
__global__ void ensemble_stats_kernel(const float* __restrict__ Ys, int members, int count, long long zY,
                                      float* __restrict__ mean, float* __restrict__ spread) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int m = 0; m < members; ++m) s += Ys[(size_t)m * zY + i];
        const float mu = s / members;
        float q = 0.f;
        for (int m = 0; m < members; ++m) {
            const float d = Ys[(size_t)m * zY + i] - mu;
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
    float* grads;   // [members][n_params]
    float* adam_m;  // [members][n_params]
    float* adam_v;
    int adam_t[64];
    float* acts;     // [layer input 0..L][members][cap_rows][width]
    float* dbuf[2];  // gradient ping-pong buffers, [members][cap_rows][width]
    int cap_rows;    // rows per member the activation buffers hold
    double* d_loss;
    int* d_err;      // set by a GEMM whose wait for the tensor cores ran out
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

// elements between two members' buffers of one layer
long long member_stride(const lbm_surrogate* s) { return (long long)s->cap_rows * (long long)act_width(s); }

// activation buffer of layer input l (l = 0: network input, L: output) of member z
float* act(lbm_surrogate* s, int l, int z) {
    return s->acts + ((size_t)l * s->cfg.n_members + z) * (size_t)member_stride(s);
}
float* dbuf(lbm_surrogate* s, int i, int z) { return s->dbuf[i] + (size_t)z * (size_t)member_stride(s); }

int ensure_rows(lbm_surrogate* s, int rows) {
    if (rows <= s->cap_rows) return LBM_OK;
    cudaFree(s->acts);
    cudaFree(s->dbuf[0]);
    cudaFree(s->dbuf[1]);
    s->acts = s->dbuf[0] = s->dbuf[1] = nullptr;
    s->cap_rows = 0;
    const size_t per = (size_t)rows * act_width(s) * s->cfg.n_members;
    SUR_CUDA(cudaMalloc(&s->acts, sizeof(float) * s->sizes.size() * per));
    SUR_CUDA(cudaMalloc(&s->dbuf[0], sizeof(float) * per));
    SUR_CUDA(cudaMalloc(&s->dbuf[1], sizeof(float) * per));
    s->cap_rows = rows;
    return LBM_OK;
}

// rows per member that one predict chunk processes: activations of every layer and
// member for a chunk stay within about 512 MB
int predict_chunk(const lbm_surrogate* s) {
    const double per_row = 4.0 * act_width(s) * s->cfg.n_members * (s->sizes.size() + 2);
    return (int)std::max(128.0, std::min(16384.0, std::floor(512.0 * 1024 * 1024 / per_row)));
}

cudaError_t gemm(const lbm_surrogate* s, GemmArgs a, int members) {
    if (a.M < 1 || a.N < 1 || a.K < 1 || members < 1) return cudaErrorInvalidValue;
    a.err = s->d_err;
    a.wait_ns = GEMM_WAIT_NS;
    a.skip_mma = 0;
    dim3 grid((a.N + TN - 1) / TN, (a.M + TM - 1) / TM, members);
    if (s->cfg.half) gemm_kernel<__half><<<grid, GEMM_THREADS, GEMM_SMEM, s->stream>>>(a);
    else gemm_kernel<__nv_bfloat16><<<grid, GEMM_THREADS, GEMM_SMEM, s->stream>>>(a);
    return cudaGetLastError();
}

// forward of members z0 .. z0 + nz - 1 on rows already in act(s, 0, z); with
// shared_input every member reads the input of member z0
int forward(lbm_surrogate* s, int z0, int nz, int rows, bool shared_input) {
    const float* P = s->params + (size_t)z0 * s->n_params;
    const int L = (int)s->sizes.size() - 1;
    const long long ms = member_stride(s);
    for (int l = 0; l < L; ++l) {
        GemmArgs a{};
        a.A = act(s, l, z0);
        a.zA = (l == 0 && shared_input) ? 0 : ms;
        a.sam = s->sizes[l];
        a.sak = 1;
        a.B = P + s->w_off[l];  // B(k, n) = W[n][k]
        a.zB = (long long)s->n_params;
        a.sbk = 1;
        a.sbn = s->sizes[l];
        a.C = act(s, l + 1, z0);
        a.zC = ms;
        a.ldc = s->sizes[l + 1];
        a.M = rows;
        a.N = s->sizes[l + 1];
        a.K = s->sizes[l];
        a.bias = P + s->b_off[l];
        a.zBias = (long long)s->n_params;
        a.epi = l < L - 1 ? EPI_BIAS_RELU : EPI_BIAS;
        SUR_CUDA(gemm(s, a, nz));
    }
    return LBM_OK;
}

// gradients of the MSE of members z0 .. z0 + nz - 1 on rows (targets T on the
// device, member stride zT) into their blocks of s->grads; member z's batch loss is
// added to loss_acc[z * zL] (device)
int backward(lbm_surrogate* s, int z0, int nz, int rows, const float* T, long long zT, double* loss_acc,
             long long zL) {
    const float* P = s->params + (size_t)z0 * s->n_params;
    float* G = s->grads + (size_t)z0 * s->n_params;
    const long long np = (long long)s->n_params, ms = member_stride(s);
    const int L = (int)s->sizes.size() - 1;
    const int nout = s->sizes[L];
    float* dz = dbuf(s, 0, z0);
    float* dh = dbuf(s, 1, z0);
    const int count = rows * nout;
    mse_grad_kernel<<<dim3(std::min(1024, (count + 255) / 256), nz), 256, 0, s->stream>>>(
        act(s, L, z0), T, dz, count, 1.0f / (float)count, LOSS_SCALE, loss_acc, ms, zT, zL);
    SUR_CUDA(cudaGetLastError());
    for (int l = L - 1; l >= 0; --l) {
        const int in = s->sizes[l], out = s->sizes[l + 1];
        GemmArgs g{};  // dW = dZ^T H : (out x in), K = rows
        g.A = dz;
        g.zA = ms;
        g.sam = 1;
        g.sak = out;
        g.B = act(s, l, z0);
        g.zB = ms;
        g.sbk = in;
        g.sbn = 1;
        g.C = G + s->w_off[l];
        g.zC = np;
        g.ldc = in;
        g.M = out;
        g.N = in;
        g.K = rows;
        g.epi = EPI_NONE;
        SUR_CUDA(gemm(s, g, nz));
        bias_grad_kernel<<<dim3((out + 127) / 128, nz), 128, 0, s->stream>>>(dz, G + s->b_off[l], rows, out, ms, np);
        SUR_CUDA(cudaGetLastError());
        if (l > 0) {
            GemmArgs d{};  // dH = dZ W, masked by ReLU'(z_{l-1}) = [h_l > 0]
            d.A = dz;
            d.zA = ms;
            d.sam = out;
            d.sak = 1;
            d.B = P + s->w_off[l];
            d.zB = np;
            d.sbk = in;
            d.sbn = 1;
            d.C = dh;
            d.zC = ms;
            d.ldc = in;
            d.M = rows;
            d.N = in;
            d.K = out;
            d.mask = act(s, l, z0);
            d.zMask = ms;
            d.ldm = in;
            d.epi = EPI_MASK;
            SUR_CUDA(gemm(s, d, nz));
            std::swap(dz, dh);
        }
    }
    return LBM_OK;
}

int adam(lbm_surrogate* s, int z0, int nz, float lr) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    AdamCorrections cc{};
    for (int z = 0; z < nz; ++z) {
        const int t = ++s->adam_t[z0 + z];
        cc.c1[z] = 1.f - std::pow(b1, (float)t);
        cc.c2[z] = 1.f - std::pow(b2, (float)t);
    }
    const int n = (int)s->n_params;
    const size_t off = (size_t)z0 * s->n_params;
    adam_kernel<<<dim3(std::min(1024, (n + 255) / 256), nz), 256, 0, s->stream>>>(
        s->params + off, s->grads + off, s->adam_m + off, s->adam_v + off, n, lr, b1, b2, eps, cc, 1.0f / LOSS_SCALE);
    SUR_CUDA(cudaGetLastError());
    return LBM_OK;
}

// After the stream has been synchronised: LBM_ERR_TIMEOUT (and the flag cleared)
// if a GEMM gave up waiting for its MMAs.
int check_gemm_flag(lbm_surrogate* s) {
    int flag = 0;
    SUR_CUDA(cudaMemcpy(&flag, s->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (!flag) return LBM_OK;
    SUR_CUDA(cudaMemset(s->d_err, 0, sizeof(int)));
    set_error("surrogate GEMM: a wait for the tensor cores ran out");
    return LBM_ERR_TIMEOUT;
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
    if ((e = cudaMalloc(&s->grads, pb)) != cudaSuccess) return bail(sur_fail(e, "cudaMalloc"));
    if ((e = cudaMalloc(&s->d_loss, sizeof(double))) != cudaSuccess) return bail(sur_fail(e, "cudaMalloc"));
    if ((e = cudaMalloc(&s->d_err, sizeof(int))) != cudaSuccess) return bail(sur_fail(e, "cudaMalloc"));
    if ((e = cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream)) != cudaSuccess) return bail(sur_fail(e, "memset"));
    if ((e = cudaFuncSetAttribute(gemm_kernel<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(gemm_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  GEMM_SMEM)) != cudaSuccess)
        return bail(sur_fail(e, "cudaFuncSetAttribute"));
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
    SUR_CUDA(cudaMemcpyAsync(act(s, 0, member), X, sizeof(float) * n * s->cfg.n_in, cudaMemcpyHostToDevice,
                             s->stream));
    if (int rc = forward(s, member, 1, n, false)) return rc;
    SUR_CUDA(cudaMemcpyAsync(Y, act(s, L, member), sizeof(float) * n * s->cfg.n_out, cudaMemcpyDeviceToHost,
                             s->stream));
    SUR_CUDA(cudaStreamSynchronize(s->stream));
    return check_gemm_flag(s);
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
    SUR_CUDA(cudaMemcpyAsync(act(s, 0, member), X, sizeof(float) * n * s->cfg.n_in, cudaMemcpyHostToDevice,
                             s->stream));
    SUR_CUDA(cudaMemcpyAsync(dT, T, sizeof(float) * n * s->cfg.n_out, cudaMemcpyHostToDevice, s->stream));
    SUR_CUDA(cudaMemsetAsync(s->d_loss, 0, sizeof(double), s->stream));
    int rc = forward(s, member, 1, n, false);
    if (!rc) rc = backward(s, member, 1, n, dT, 0, s->d_loss, 0);
    cudaFreeAsync(dT, s->stream);
    if (rc) return rc;
    SUR_CUDA(cudaMemcpyAsync(grads, s->grads + (size_t)member * s->n_params, sizeof(float) * s->n_params,
                             cudaMemcpyDeviceToHost, s->stream));
    double l = 0;
    SUR_CUDA(cudaMemcpyAsync(&l, s->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    SUR_CUDA(cudaStreamSynchronize(s->stream));
    if (int rc2 = check_gemm_flag(s)) return rc2;
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
    const int nin = s->cfg.n_in, nout = s->cfg.n_out, M = s->cfg.n_members;
    const int E = std::max(1, epochs);
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
    TR_CUDA(cudaMalloc(&dTb, sizeof(float) * (size_t)M * batch * nout));
    TR_CUDA(cudaMalloc(&dIdx, sizeof(int) * (size_t)M * E * n));
    TR_CUDA(cudaMalloc(&dLoss, sizeof(double) * (size_t)M * E));
    TR_CUDA(cudaMemcpyAsync(dX, X, sizeof(float) * (size_t)n * nin, cudaMemcpyHostToDevice, s->stream));
    TR_CUDA(cudaMemcpyAsync(dT, T, sizeof(float) * (size_t)n * nout, cudaMemcpyHostToDevice, s->stream));
    TR_CUDA(cudaMemsetAsync(dLoss, 0, sizeof(double) * (size_t)M * E, s->stream));
    // seeded Fisher-Yates order per member and epoch, [member][epoch][n]
    std::vector<int> order((size_t)M * E * n);
    for (int m = 0; m < M; ++m) {
        uint64_t st = shuffle_seed * 0x9E3779B97F4A7C15ull + (uint64_t)m * 0xD1B54A32D192ED03ull + 7;
        for (int ep = 0; ep < epochs; ++ep) {
            int* o = order.data() + ((size_t)m * E + ep) * n;
            for (int i = 0; i < n; ++i) o[i] = i;
            for (int i = n - 1; i > 0; --i) std::swap(o[i], o[splitmix(st) % (uint64_t)(i + 1)]);
        }
    }
    TR_CUDA(cudaMemcpyAsync(dIdx, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice, s->stream));
    // every member steps through its own order at once: one launch per layer and pass
    const long long ms = member_stride(s);
    for (int ep = 0; ep < epochs; ++ep) {
        for (int b0 = 0; b0 + batch <= n; b0 += batch) {
            const int* idx = dIdx + (size_t)ep * n + b0;
            gather_rows_kernel<<<dim3(std::min(1024, (batch * nin + 255) / 256), M), 256, 0, s->stream>>>(
                dX, idx, act(s, 0, 0), batch, nin, (long long)E * n, ms);
            gather_rows_kernel<<<dim3(std::min(1024, (batch * nout + 255) / 256), M), 256, 0, s->stream>>>(
                dT, idx, dTb, batch, nout, (long long)E * n, (long long)batch * nout);
            TR_CUDA(cudaGetLastError());
            int rc = forward(s, 0, M, batch, false);
            if (!rc) rc = backward(s, 0, M, batch, dTb, (long long)batch * nout, dLoss + ep, E);
            if (!rc) rc = adam(s, 0, M, lr);
            if (rc) {
                cleanup();
                return rc;
            }
        }
    }
    if (epoch_loss && epochs > 0) {
        TR_CUDA(cudaMemcpyAsync(epoch_loss, dLoss, sizeof(double) * (size_t)M * epochs, cudaMemcpyDeviceToHost,
                                s->stream));
    }
    TR_CUDA(cudaStreamSynchronize(s->stream));
    // per-epoch loss = mean over batches of the batch MSE
    if (epoch_loss) {
        const int nb = n / batch;
        for (int i = 0; i < M * epochs; ++i) epoch_loss[i] /= std::max(1, nb);
    }
    cleanup();
#undef TR_CUDA
    return check_gemm_flag(s);
}

int lbm_surrogate_predict(lbm_surrogate* s, const float* X, int n, float* mean, float* spread) {
    if (!s || !X || !mean || !spread || n < 1) {
        set_error("lbm_surrogate_predict: bad argument");
        return LBM_ERR_ARG;
    }
    const int nin = s->cfg.n_in, nout = s->cfg.n_out, M = s->cfg.n_members, L = (int)s->sizes.size() - 1;
    const int chunk = std::min(n, predict_chunk(s));
    if (int rc = ensure_rows(s, chunk)) return rc;
    float *dMean = nullptr, *dSpread = nullptr;
    auto cleanup = [&]() { cudaFree(dMean); cudaFree(dSpread); };
    cudaError_t e;
    if ((e = cudaMalloc(&dMean, sizeof(float) * (size_t)chunk * nout)) != cudaSuccess) { cleanup(); return sur_fail(e, "cudaMalloc"); }
    if ((e = cudaMalloc(&dSpread, sizeof(float) * (size_t)chunk * nout)) != cudaSuccess) { cleanup(); return sur_fail(e, "cudaMalloc"); }
    for (int r0 = 0; r0 < n; r0 += chunk) {
        const int rows = std::min(chunk, n - r0);
        if ((e = cudaMemcpyAsync(act(s, 0, 0), X + (size_t)r0 * nin, sizeof(float) * rows * nin, cudaMemcpyHostToDevice,
                                 s->stream)) != cudaSuccess) { cleanup(); return sur_fail(e, "cudaMemcpyAsync"); }
        // all members in one launch per layer, all reading the one copy of the input
        if (int rc = forward(s, 0, M, rows, true)) { cleanup(); return rc; }
        ensemble_stats_kernel<<<std::min(1024, (rows * nout + 255) / 256), 256, 0, s->stream>>>(
            act(s, L, 0), M, rows * nout, member_stride(s), dMean, dSpread);
        if ((e = cudaGetLastError()) != cudaSuccess) { cleanup(); return sur_fail(e, "ensemble_stats_kernel"); }
        if ((e = cudaMemcpyAsync(mean + (size_t)r0 * nout, dMean, sizeof(float) * rows * nout, cudaMemcpyDeviceToHost,
                                 s->stream)) != cudaSuccess) { cleanup(); return sur_fail(e, "copy"); }
        if ((e = cudaMemcpyAsync(spread + (size_t)r0 * nout, dSpread, sizeof(float) * rows * nout,
                                 cudaMemcpyDeviceToHost, s->stream)) != cudaSuccess) { cleanup(); return sur_fail(e, "copy"); }
        if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) { cleanup(); return sur_fail(e, "sync"); }
    }
    cleanup();
    return check_gemm_flag(s);
}

int lbm_surrogate_selftest_wait(int limit_us, int* gave_up) {
    if (!gave_up || limit_us < 1 || limit_us > 10000000) {
        set_error("lbm_surrogate_selftest_wait: limit_us in [1, 1e7] and a result pointer");
        return LBM_ERR_ARG;
    }
    *gave_up = 0;
    float* buf = nullptr;
    int* d_flag = nullptr;
    SUR_CUDA(cudaMalloc(&buf, sizeof(float) * 4));
    cudaError_t e = cudaMalloc(&d_flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(buf, 0, sizeof(float) * 4);
    if (e == cudaSuccess) e = cudaMemset(d_flag, 0, sizeof(int));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gemm_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM);
    if (e == cudaSuccess) {
        GemmArgs a{};
        a.A = buf;
        a.B = buf + 1;
        a.C = buf + 2;
        a.M = a.N = a.K = 1;
        a.sam = a.sak = a.sbk = a.sbn = a.ldc = 1;
        a.epi = EPI_NONE;
        a.err = d_flag;
        a.wait_ns = 1000ull * (unsigned long long)limit_us;
        a.skip_mma = 1;  // no MMA and no commit: the completion barrier never completes
        gemm_kernel<__nv_bfloat16><<<1, GEMM_THREADS, GEMM_SMEM>>>(a);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(buf);
    cudaFree(d_flag);
    if (e != cudaSuccess) return sur_fail(e, "lbm_surrogate_selftest_wait");
    *gave_up = flag != 0;
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
    cudaFree(s->d_err);
    delete s;
}

}  // extern "C"
