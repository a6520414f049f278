// sbr_surrogate.cu -- learned surrogate of the SBR field: a Fourier-feature MLP
// in BF16 with FP32 accumulation whose forward and backward products run on
// the tcgen05 tensor-core GEMM of sbr_gemm.cu.
//
// Network (per ensemble member): input (az, el, f) -> (sin az, cos az, el / 30
// deg, log-frequency mapped to [-1, 1]) -> Fourier features [sin 2 pi B x,
// cos 2 pi B x] (B fixed, N(0, sigma^2)) -> depth x (width GELU) -> 4 outputs
// (Re and Im of HH and VV, divided by a target scale). Hidden layers: BF16
// activations and weights, FP32 accumulation (tcgen05 GEMM), FP32 master weights
// with Adam. The 4-output head runs on CUDA cores.
//
// One training step on a batch of M samples (M a multiple of 128):
//   forward  h0 = FF(x); z_l = h_l W_l^T + b_l, h_{l+1} = GELU(z_l)   (GEMM, fused epilogue)
//            y = h_D W_h^T + b_h                                        (head kernel)
//   loss     mean squared error over the 4 outputs
//   backward dz_{D-1} = (dy W_h) * GELU'(z_{D-1});
//            dW_l = dz_l^T h_l (GEMM on transposed operands), db_l = sum_m dz_l
//            dz_{l-1} = (dz_l W_l) * GELU'(z_{l-1})                     (GEMM with W_l^T, fused epilogue)
//   Adam on all FP32 parameters, then BF16 copies of W_l and W_l^T refreshed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <random>
#include <string>
#include <vector>

#include "sbr.h"
#include "sbr_internal.h"

using namespace sbr;

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxDepth = 16;
constexpr int kOut = 4;
constexpr int kIn = 4;

std::mutex g_gemm_mu;
int* g_gemm_err[64] = {nullptr};

// ---------------------------------------------------------------- small kernels
// raw (az deg, el deg, f Hz) -> the 4 network inputs
__global__ void k_encode(const double* raw, int n, float* x4)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double az = raw[3 * i] * (kPi / 180.0), el = raw[3 * i + 1], f = raw[3 * i + 2];
    x4[4 * i + 0] = (float)sin(az);
    x4[4 * i + 1] = (float)cos(az);
    x4[4 * i + 2] = (float)(el / 30.0);
    x4[4 * i + 3] = (float)(2.0 * (log(f / 1e9) / log(12.0)) - 1.0);
}

__global__ void k_gather(const float* x4, const float* y4, const int* idx, int n, float* xb, float* yb)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = idx[i];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        xb[4 * i + c] = x4[4 * (size_t)j + c];
        if (yb) yb[4 * i + c] = y4[4 * (size_t)j + c];
    }
}

// Fourier features: h0[m][j] = sin(2 pi B_j . x_m) (j < nf/2), cos(...) (j >= nf/2)
__global__ void k_fourier(const float* x4, const float* B, int M, int nh, __nv_bfloat16* h0)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)M * nh) return;
    const int m = (int)(i / nh), j = (int)(i % nh);
    const float* b = B + 4 * j;
    const float* x = x4 + 4 * m;
    const float arg = b[0] * x[0] + b[1] * x[1] + b[2] * x[2] + b[3] * x[3];
    float s, c;
    sincospif(2.f * arg, &s, &c);
    h0[(size_t)m * (2 * nh) + j] = __float2bfloat16_rn(s);
    h0[(size_t)m * (2 * nh) + nh + j] = __float2bfloat16_rn(c);
}

__device__ __forceinline__ float gelu_grad_f(float z)
{
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.3989422804014327f * expf(-0.5f * z * z);
}

// head: y[m][o] = sum_k h[m][k] W[o][k] + b[o]; one warp per row
__global__ void k_head_fwd(const __nv_bfloat16* h, int M, int K, const float* W, const float* b, float* y)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= M) return;
    float acc[kOut] = {0.f, 0.f, 0.f, 0.f};
    for (int k = lane; k < K; k += 32) {
        const float v = __bfloat162float(h[(size_t)warp * K + k]);
#pragma unroll
        for (int o = 0; o < kOut; ++o) acc[o] = fmaf(v, W[o * K + k], acc[o]);
    }
#pragma unroll
    for (int o = 0; o < kOut; ++o)
        for (int s = 16; s > 0; s >>= 1) acc[o] += __shfl_xor_sync(0xffffffffu, acc[o], s);
    if (lane == 0)
#pragma unroll
        for (int o = 0; o < kOut; ++o) y[(size_t)warp * kOut + o] = acc[o] + b[o];
}

// dy = 2 (y - t) / (M * 4); loss sum in FP64
__global__ void k_loss(const float* y, const float* t, int n, float* dy, double* loss)
{
    __shared__ double s_red[8];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (i < n) {
        const float d = y[i] - t[i];
        dy[i] = 2.f * d / (float)n;
        l = (double)d * d;
    }
    for (int s = 16; s > 0; s >>= 1) l += __shfl_xor_sync(0xffffffffu, l, s);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t2 += s_red[w];
        atomicAdd(loss, t2);
    }
}

// dz[m][k] = (sum_o dy[m][o] W[o][k]) * gelu'(z[m][k])
__global__ void k_head_bwd_dz(const float* dy, const float* W, const float* z, int M, int K, __nv_bfloat16* dz)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)M * K) return;
    const int m = (int)(i / K), k = (int)(i % K);
    float s = 0.f;
#pragma unroll
    for (int o = 0; o < kOut; ++o) s = fmaf(dy[m * kOut + o], W[o * K + k], s);
    dz[i] = __float2bfloat16_rn(s * gelu_grad_f(z[i]));
}

// Column sums over the batch in two fixed-order stages (deterministic): stage 1
// gives one partial per kRedRows rows (block 32 columns x 8 row lanes), stage 2
// adds the partials in order.
constexpr int kRedRows = 256;

// head gradient, stage 1: part[p][o][k] = sum over rows m of chunk p of dy[m][o] h[m][k]
// (k < K) and of dy[m][o] (k = K, the bias)
__global__ void k_head_dw_part(const float* dy, const __nv_bfloat16* h, int M, int K, float* part)
{
    __shared__ float sh[8][kOut][33];
    const int k = blockIdx.x * 32 + threadIdx.x, p = blockIdx.y;
    float acc[kOut] = {0.f, 0.f, 0.f, 0.f};
    if (k <= K) {
        const int r1 = min(M, (p + 1) * kRedRows);
#pragma unroll 4
        for (int m = p * kRedRows + threadIdx.y; m < r1; m += 8) {
            const float v = k < K ? __bfloat162float(h[(size_t)m * K + k]) : 1.f;
#pragma unroll
            for (int o = 0; o < kOut; ++o) acc[o] = fmaf(dy[m * kOut + o], v, acc[o]);
        }
    }
#pragma unroll
    for (int o = 0; o < kOut; ++o) sh[threadIdx.y][o][threadIdx.x] = acc[o];
    __syncthreads();
    if (threadIdx.y < kOut && k <= K) {
        const int o = threadIdx.y;
        float t = 0.f;
        for (int y = 0; y < 8; ++y) t += sh[y][o][threadIdx.x];
        part[((size_t)p * kOut + o) * (K + 1) + k] = t;
    }
}

// head gradient, stage 2: dW[o][k], db[o] = sum over the P partials
__global__ void k_head_dw_fin(const float* part, int P, int K, float* dW, float* db)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= kOut * (K + 1)) return;
    const int o = j / (K + 1), k = j % (K + 1);
    float t = 0.f;
    for (int q = 0; q < P; ++q) t += part[((size_t)q * kOut + o) * (K + 1) + k];
    if (k < K) dW[o * K + k] = t;
    else db[o] = t;
}

// bias gradient, stage 1: part[p][n] = sum over rows m of chunk p of dz[m][n]
__global__ void k_colsum_part(const __nv_bfloat16* dz, int M, int N, float* part)
{
    __shared__ float sh[8][33];
    const int n = blockIdx.x * 32 + threadIdx.x, p = blockIdx.y;
    float acc = 0.f;
    if (n < N) {
        const int r1 = min(M, (p + 1) * kRedRows);
#pragma unroll 4
        for (int m = p * kRedRows + threadIdx.y; m < r1; m += 8) acc += __bfloat162float(dz[(size_t)m * N + n]);
    }
    sh[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.y == 0 && n < N) {
        float t = 0.f;
        for (int y = 0; y < 8; ++y) t += sh[y][threadIdx.x];
        part[(size_t)p * N + n] = t;
    }
}

// bias gradient, stage 2
__global__ void k_colsum_fin(const float* part, int P, int N, float* db)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float t = 0.f;
    for (int q = 0; q < P; ++q) t += part[(size_t)q * N + n];
    db[n] = t;
}

// out[c][r] = in[r][c] for a [R x Cc] BF16 matrix, 32 x 32 tiles through shared memory
__global__ void k_transpose(const __nv_bfloat16* in, int R, int Cc, __nv_bfloat16* out)
{
    __shared__ __nv_bfloat16 t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = r0 + y, c = c0 + threadIdx.x;
        if (r < R && c < Cc) t[y][threadIdx.x] = in[(size_t)r * Cc + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int c = c0 + y, r = r0 + threadIdx.x;
        if (r < R && c < Cc) out[(size_t)c * R + r] = t[threadIdx.x][y];
    }
}

__global__ void k_adam(float* p, float* m, float* v, const float* g, long long n, float lr, float b1, float b2,
                       float c1, float c2, float eps)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

__global__ void k_to_bf16(const float* in, long long n, __nv_bfloat16* out)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16_rn(in[i]);
}

// ensemble mean (scaled back) and spread: per point, max over HH and VV of the
// range over members of 10 log10 |E|^2
__global__ void k_ens_stats(const float* y, int n_members, long long stride, int n, float scale, double* mean,
                            float* spread)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float mu[kOut] = {0.f, 0.f, 0.f, 0.f};
    float lo[2] = {1e30f, 1e30f}, hi[2] = {-1e30f, -1e30f};
    for (int e = 0; e < n_members; ++e) {
        const float* r = y + e * stride + (size_t)i * kOut;
#pragma unroll
        for (int o = 0; o < kOut; ++o) mu[o] += r[o];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const float a2 = r[2 * p] * r[2 * p] + r[2 * p + 1] * r[2 * p + 1];
            const float db = 10.f * log10f(fmaxf(a2, 1e-30f));
            lo[p] = fminf(lo[p], db);
            hi[p] = fmaxf(hi[p], db);
        }
    }
#pragma unroll
    for (int o = 0; o < kOut; ++o) mean[(size_t)i * kOut + o] = (double)(mu[o] / n_members) * scale;
    spread[i] = fmaxf(hi[0] - lo[0], hi[1] - lo[1]);
}

inline unsigned blocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ------------------------------------------------------------------ surrogate state
struct sbr_surrogate {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    sbr_surrogate_opts opt;
    std::string err;
    int nh = 0;  // Fourier frequencies (features = 2 nh)
    std::vector<int> K, N;  // hidden layer l: N[l] x K[l]
    std::vector<long long> offW, offb;  // offsets in the flat parameter vector (layer depth = head)
    long long n_params = 0;
    long long offWbf_total = 0;
    std::vector<long long> offWbf;  // offsets of the BF16 copies
    // per member, device
    std::vector<float*> P, Pm, Pv, Bf;  // parameters, Adam moments, Fourier matrices
    std::vector<__nv_bfloat16*> Wbf, WTbf;
    std::vector<long long> steps;
    float* G = nullptr;  // gradient (shared by members)
    // activations for batches of up to cap rows
    int cap = 0;
    std::vector<__nv_bfloat16*> h;   // h[0..depth] BF16 [cap x width_l]
    std::vector<float*> z;           // z[0..depth-1] FP32 [cap x N_l]
    std::vector<__nv_bfloat16*> dz;  // dz[l] BF16 [cap x N_l]
    __nv_bfloat16 *dzT = nullptr, *hT = nullptr;
    float *y = nullptr, *dy = nullptr, *xb = nullptr, *yb = nullptr;
    float* red = nullptr;  // partial column sums [cap / 256 x 4 (width + 1)]
    double* loss = nullptr;
    int* gerr = nullptr;
    int* idx = nullptr;
    float target_scale = 1.f;
    bool trained = false;
};

namespace {

int sfail(sbr_surrogate* s, int code, const char* msg)
{
    if (s) s->err = msg;
    return code;
}

#define SCK(call, what)                                                                   \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            cudaGetLastError();                                                           \
            return sfail(s, e_ == cudaErrorMemoryAllocation ? SBR_ERR_OOM : SBR_ERR_CUDA, \
                         (std::string(what) + ": " + cudaGetErrorString(e_)).c_str());    \
        }                                                                                 \
    } while (0)

int ensure_cap(sbr_surrogate* s, int M)
{
    if (M <= s->cap) return SBR_OK;
    const int D = s->opt.depth;
    auto fr = [](void* p) {
        if (p) cudaFree(p);
    };
    for (auto p : s->h) fr(p);
    for (auto p : s->z) fr(p);
    for (auto p : s->dz) fr(p);
    fr(s->dzT);
    fr(s->hT);
    fr(s->y);
    fr(s->dy);
    fr(s->xb);
    fr(s->yb);
    fr(s->idx);
    fr(s->red);
    s->h.assign(D + 1, nullptr);
    s->z.assign(D, nullptr);
    s->dz.assign(D, nullptr);
    const int wmax = std::max(s->opt.width, s->opt.n_fourier);
    for (int l = 0; l <= D; ++l) SCK(cudaMalloc(&s->h[l], sizeof(__nv_bfloat16) * (size_t)M * (l == 0 ? s->opt.n_fourier : s->opt.width)), "alloc h");
    for (int l = 0; l < D; ++l) {
        SCK(cudaMalloc(&s->z[l], sizeof(float) * (size_t)M * s->opt.width), "alloc z");
        SCK(cudaMalloc(&s->dz[l], sizeof(__nv_bfloat16) * (size_t)M * s->opt.width), "alloc dz");
    }
    SCK(cudaMalloc(&s->dzT, sizeof(__nv_bfloat16) * (size_t)M * s->opt.width), "alloc dzT");
    SCK(cudaMalloc(&s->hT, sizeof(__nv_bfloat16) * (size_t)M * wmax), "alloc hT");
    SCK(cudaMalloc(&s->y, sizeof(float) * (size_t)M * kOut * std::max(1, s->opt.n_members)), "alloc y");
    SCK(cudaMalloc(&s->dy, sizeof(float) * (size_t)M * kOut), "alloc dy");
    SCK(cudaMalloc(&s->xb, sizeof(float) * (size_t)M * kIn), "alloc xb");
    SCK(cudaMalloc(&s->yb, sizeof(float) * (size_t)M * kOut), "alloc yb");
    SCK(cudaMalloc(&s->idx, sizeof(int) * (size_t)M), "alloc idx");
    SCK(cudaMalloc(&s->red, sizeof(float) * (size_t)((M + kRedRows - 1) / kRedRows) * kOut * (wmax + 1)),
        "alloc partial sums");
    s->cap = M;
    return SBR_OK;
}

// refresh the BF16 copies of W_l and W_l^T of member e
int refresh_bf16(sbr_surrogate* s, int e)
{
    for (int l = 0; l < s->opt.depth; ++l) {
        const long long n = (long long)s->N[l] * s->K[l];
        __nv_bfloat16* w = s->Wbf[e] + s->offWbf[l];
        k_to_bf16<<<blocks(n, 256), 256, 0, s->stream>>>(s->P[e] + s->offW[l], n, w);
        dim3 g((s->K[l] + 31) / 32, (s->N[l] + 31) / 32);
        k_transpose<<<g, dim3(32, 8), 0, s->stream>>>(w, s->N[l], s->K[l], s->WTbf[e] + s->offWbf[l]);
    }
    SCK(cudaGetLastError(), "refresh weights");
    return SBR_OK;
}

// forward pass of member e on xb[0..M): fills h, z and y (at y + yoff)
// keep_z: store the FP32 pre-activations for a backward pass (prediction writes only the BF16 activations)
int forward(sbr_surrogate* s, int e, int M, float* yout, bool keep_z = true)
{
    const int D = s->opt.depth;
    k_fourier<<<blocks((long long)M * s->nh, 256), 256, 0, s->stream>>>(s->xb, s->Bf[e], M, s->nh, s->h[0]);
    for (int l = 0; l < D; ++l) {
        GemmEpi ep;
        memset(&ep, 0, sizeof(ep));
        ep.mode = kEpiBiasGelu;
        ep.M = M;
        ep.c_f32 = keep_z ? s->z[l] : nullptr;
        ep.ldc = s->N[l];
        ep.out_bf16 = s->h[l + 1];
        ep.ldo = s->N[l];
        ep.bias = s->P[e] + s->offb[l];
        SCK(gemm_bf16_tn(s->h[l], s->K[l], s->Wbf[e] + s->offWbf[l], s->K[l], M, s->N[l], s->K[l], ep, s->gerr,
                         s->stream),
            "forward gemm");
    }
    k_head_fwd<<<blocks((long long)M * 32, 256), 256, 0, s->stream>>>(s->h[D], M, s->opt.width, s->P[e] + s->offW[D],
                                                                       s->P[e] + s->offb[D], yout);
    SCK(cudaGetLastError(), "head");
    return SBR_OK;
}

// backward pass of member e (after forward on the same batch; targets in yb): gradient in G
// The sum of squared errors is added to *lacc (zeroed first when lacc is null: s->loss).
int backward(sbr_surrogate* s, int e, int M, double* lacc = nullptr)
{
    const int D = s->opt.depth, W = s->opt.width;
    if (!lacc) {
        lacc = s->loss;
        cudaMemsetAsync(lacc, 0, sizeof(double), s->stream);
    }
    k_loss<<<blocks((long long)M * kOut, 256), 256, 0, s->stream>>>(s->y, s->yb, M * kOut, s->dy, lacc);
    const int P = (M + kRedRows - 1) / kRedRows;
    k_head_dw_part<<<dim3((W + 1 + 31) / 32, P), dim3(32, 8), 0, s->stream>>>(s->dy, s->h[D], M, W, s->red);
    k_head_dw_fin<<<blocks(kOut * (W + 1), 256), 256, 0, s->stream>>>(s->red, P, W, s->G + s->offW[D],
                                                                        s->G + s->offb[D]);
    k_head_bwd_dz<<<blocks((long long)M * W, 256), 256, 0, s->stream>>>(s->dy, s->P[e] + s->offW[D], s->z[D - 1], M, W,
                                                                         s->dz[D - 1]);
    for (int l = D - 1; l >= 0; --l) {
        // dW_l = dz_l^T h_l : A = dz_l^T [N x M], B = h_l^T [K x M]
        dim3 g1((s->N[l] + 31) / 32, (M + 31) / 32), g2((s->K[l] + 31) / 32, (M + 31) / 32);
        k_transpose<<<g1, dim3(32, 8), 0, s->stream>>>(s->dz[l], M, s->N[l], s->dzT);
        k_transpose<<<g2, dim3(32, 8), 0, s->stream>>>(s->h[l], M, s->K[l], s->hT);
        GemmEpi ep;
        memset(&ep, 0, sizeof(ep));
        ep.mode = kEpiF32;
        ep.M = s->N[l];
        ep.c_f32 = s->G + s->offW[l];
        ep.ldc = s->K[l];
        SCK(gemm_bf16_tn(s->dzT, M, s->hT, M, s->N[l], s->K[l], M, ep, s->gerr, s->stream), "weight-gradient gemm");
        k_colsum_part<<<dim3((s->N[l] + 31) / 32, P), dim3(32, 8), 0, s->stream>>>(s->dz[l], M, s->N[l], s->red);
        k_colsum_fin<<<blocks(s->N[l], 256), 256, 0, s->stream>>>(s->red, P, s->N[l], s->G + s->offb[l]);
        if (l > 0) {
            // dz_{l-1} = (dz_l W_l) * gelu'(z_{l-1}) : A = dz_l [M x N], B = W_l^T [K x N]
            GemmEpi eg;
            memset(&eg, 0, sizeof(eg));
            eg.mode = kEpiGeluGrad;
            eg.M = M;
            eg.out_bf16 = s->dz[l - 1];
            eg.ldo = s->K[l];
            eg.z = s->z[l - 1];
            eg.ldz = s->K[l];
            SCK(gemm_bf16_tn(s->dz[l], s->N[l], s->WTbf[e] + s->offWbf[l], s->N[l], M, s->K[l], s->N[l], eg, s->gerr,
                             s->stream),
                "input-gradient gemm");
        }
    }
    SCK(cudaGetLastError(), "backward");
    return SBR_OK;
}

int check_gemm_err(sbr_surrogate* s)
{
    int herr = 0;
    SCK(cudaMemcpyAsync(&herr, s->gerr, sizeof(int), cudaMemcpyDeviceToHost, s->stream), "copy error flag");
    SCK(cudaStreamSynchronize(s->stream), "sync");
    if (herr) return sfail(s, SBR_ERR_TIMEOUT, "tensor-core GEMM: a bounded wait gave up");
    return SBR_OK;
}

int upload_inputs(sbr_surrogate* s, const double* x, int64_t n, float** x4)
{
    double* raw = nullptr;
    SCK(cudaMalloc(&raw, sizeof(double) * 3 * (size_t)n), "alloc inputs");
    SCK(cudaMalloc(x4, sizeof(float) * kIn * (size_t)n), "alloc inputs");
    cudaError_t e = cudaMemcpyAsync(raw, x, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) {
        k_encode<<<blocks(n, 256), 256, 0, s->stream>>>(raw, (int)n, *x4);
        e = cudaStreamSynchronize(s->stream);
    }
    cudaFree(raw);
    SCK(e, "encode inputs");
    return SBR_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI
extern "C" {

int sbr_gemm_bf16_tn(const void* A, int lda, const void* B, int ldb, int M, int N, int K, float* C, int ldc,
                     void* cuda_stream)
{
    if (!A || !B || !C) return SBR_ERR_ARG;
    if (!gemm_shape_ok(M, N, K) || lda < K || ldb < K || ldc < N || lda % 8 || ldb % 8 || ldc % 4)
        return SBR_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SBR_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_gemm_mu);
    if (!g_gemm_err[dev]) {
        if (cudaMalloc(&g_gemm_err[dev], sizeof(int)) != cudaSuccess) return SBR_ERR_OOM;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (cudaMemsetAsync(g_gemm_err[dev], 0, sizeof(int), st) != cudaSuccess) return SBR_ERR_CUDA;
    GemmEpi ep;
    memset(&ep, 0, sizeof(ep));
    ep.mode = kEpiF32;
    ep.M = M;
    ep.c_f32 = C;
    ep.ldc = ldc;
    if (gemm_bf16_tn(A, lda, B, ldb, M, N, K, ep, g_gemm_err[dev], st) != cudaSuccess) return SBR_ERR_CUDA;
    int herr = 0;
    if (cudaMemcpyAsync(&herr, g_gemm_err[dev], sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return SBR_ERR_CUDA;
    return herr ? SBR_ERR_TIMEOUT : SBR_OK;
}

int sbr_gemm_bf16_tn_async(const void* A, int lda, const void* B, int ldb, int M, int N, int K, float* C, int ldc,
                           int* err_dev, void* cuda_stream)
{
    if (!A || !B || !C || !err_dev) return SBR_ERR_ARG;
    if (!gemm_shape_ok(M, N, K) || lda < K || ldb < K || ldc < N || lda % 8 || ldb % 8 || ldc % 4)
        return SBR_ERR_ARG;
    GemmEpi ep;
    memset(&ep, 0, sizeof(ep));
    ep.mode = kEpiF32;
    ep.M = M;
    ep.c_f32 = C;
    ep.ldc = ldc;
    return gemm_bf16_tn(A, lda, B, ldb, M, N, K, ep, err_dev, (cudaStream_t)cuda_stream) == cudaSuccess ? SBR_OK
                                                                                                      : SBR_ERR_CUDA;
}

const char* sbr_surrogate_last_error(const sbr_surrogate* s) { return s ? s->err.c_str() : ""; }

int sbr_surrogate_create(sbr_surrogate** out, int device, void* cuda_stream, const sbr_surrogate_opts* opt)
{
    if (!out) return SBR_ERR_ARG;
    *out = nullptr;
    sbr_surrogate_opts o;
    o.n_members = 4;
    o.width = 512;
    o.depth = 6;
    o.n_fourier = 256;
    o.fourier_sigma = 4.f;
    o.seed = 1;
    if (opt) o = *opt;
    if (o.n_members < 1 || o.n_members > 16 || o.width < 128 || o.width % 128 || o.depth < 1 || o.depth > kMaxDepth ||
        o.n_fourier < 128 || o.n_fourier % 128 || !(o.fourier_sigma > 0.f))
        return SBR_ERR_ARG;
    int nd = 0;
    if (cudaGetDeviceCount(&nd) != cudaSuccess || nd == 0) {
        cudaGetLastError();
        return SBR_ERR_NODEV;
    }
    if (device < 0 || device >= nd || cudaSetDevice(device) != cudaSuccess) return SBR_ERR_ARG;
    sbr_surrogate* s = new sbr_surrogate();
    s->device = device;
    s->opt = o;
    s->nh = o.n_fourier / 2;
    if (cuda_stream) {
        s->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete s;
            return SBR_ERR_CUDA;
        }
        s->own_stream = true;
    }
    const int D = o.depth;
    s->K.resize(D);
    s->N.resize(D);
    for (int l = 0; l < D; ++l) {
        s->K[l] = l == 0 ? o.n_fourier : o.width;
        s->N[l] = o.width;
    }
    long long off = 0, offbf = 0;
    for (int l = 0; l <= D; ++l) {
        const int Kl = l < D ? s->K[l] : o.width, Nl = l < D ? s->N[l] : kOut;
        s->offW.push_back(off);
        off += (long long)Nl * Kl;
        s->offb.push_back(off);
        off += Nl;
        if (l < D) {
            s->offWbf.push_back(offbf);
            offbf += (long long)Nl * Kl;
        }
    }
    s->n_params = off;
    s->offWbf_total = offbf;
    // parameters: He-normal hidden layers, small head, zero biases; Fourier matrix N(0, sigma^2)
    std::mt19937_64 rng(o.seed);
    std::normal_distribution<float> nd01(0.f, 1.f);
    std::vector<float> hp((size_t)off), hb((size_t)4 * s->nh);
    int rc = SBR_OK;
    for (int e = 0; e < o.n_members && rc == SBR_OK; ++e) {
        std::fill(hp.begin(), hp.end(), 0.f);
        for (int l = 0; l <= D; ++l) {
            const int Kl = l < D ? s->K[l] : o.width, Nl = l < D ? s->N[l] : kOut;
            const float sd = l < D ? sqrtf(2.f / (float)Kl) : sqrtf(1.f / (float)Kl);
            for (long long i = 0; i < (long long)Nl * Kl; ++i) hp[(size_t)(s->offW[l] + i)] = sd * nd01(rng);
        }
        for (auto& v : hb) v = o.fourier_sigma * nd01(rng);
        float *P, *Pm, *Pv, *Bf;
        __nv_bfloat16 *Wb, *WTb;
        if (cudaMalloc(&P, sizeof(float) * off) != cudaSuccess || cudaMalloc(&Pm, sizeof(float) * off) != cudaSuccess ||
            cudaMalloc(&Pv, sizeof(float) * off) != cudaSuccess ||
            cudaMalloc(&Bf, sizeof(float) * hb.size()) != cudaSuccess ||
            cudaMalloc(&Wb, sizeof(__nv_bfloat16) * offbf) != cudaSuccess ||
            cudaMalloc(&WTb, sizeof(__nv_bfloat16) * offbf) != cudaSuccess) {
            rc = SBR_ERR_OOM;
            break;
        }
        s->P.push_back(P);
        s->Pm.push_back(Pm);
        s->Pv.push_back(Pv);
        s->Bf.push_back(Bf);
        s->Wbf.push_back(Wb);
        s->WTbf.push_back(WTb);
        s->steps.push_back(0);
        cudaMemcpy(P, hp.data(), sizeof(float) * off, cudaMemcpyHostToDevice);
        cudaMemcpy(Bf, hb.data(), sizeof(float) * hb.size(), cudaMemcpyHostToDevice);
        cudaMemset(Pm, 0, sizeof(float) * off);
        cudaMemset(Pv, 0, sizeof(float) * off);
        rc = refresh_bf16(s, e);
    }
    if (rc == SBR_OK && (cudaMalloc(&s->G, sizeof(float) * off) != cudaSuccess ||
                         cudaMalloc(&s->loss, sizeof(double)) != cudaSuccess ||
                         cudaMalloc(&s->gerr, sizeof(int)) != cudaSuccess))
        rc = SBR_ERR_OOM;
    if (rc == SBR_OK && cudaMemsetAsync(s->gerr, 0, sizeof(int), s->stream) != cudaSuccess) rc = SBR_ERR_CUDA;
    if (rc == SBR_OK && cudaStreamSynchronize(s->stream) != cudaSuccess) rc = SBR_ERR_CUDA;
    if (rc != SBR_OK) {
        sbr_surrogate_destroy(s);
        return rc;
    }
    *out = s;
    return SBR_OK;
}

void sbr_surrogate_destroy(sbr_surrogate* s)
{
    if (!s) return;
    cudaSetDevice(s->device);
    cudaStreamSynchronize(s->stream);
    auto fr = [](void* p) {
        if (p) cudaFree(p);
    };
    for (auto p : s->P) fr(p);
    for (auto p : s->Pm) fr(p);
    for (auto p : s->Pv) fr(p);
    for (auto p : s->Bf) fr(p);
    for (auto p : s->Wbf) fr(p);
    for (auto p : s->WTbf) fr(p);
    for (auto p : s->h) fr(p);
    for (auto p : s->z) fr(p);
    for (auto p : s->dz) fr(p);
    fr(s->G);
    fr(s->dzT);
    fr(s->hT);
    fr(s->y);
    fr(s->dy);
    fr(s->xb);
    fr(s->yb);
    fr(s->loss);
    fr(s->gerr);
    fr(s->idx);
    fr(s->red);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
}

int64_t sbr_surrogate_num_params(const sbr_surrogate* s) { return s ? s->n_params : 0; }

int sbr_surrogate_params(sbr_surrogate* s, int member, float* get, const float* set)
{
    if (!s || member < 0 || member >= s->opt.n_members) return SBR_ERR_ARG;
    SCK(cudaSetDevice(s->device), "cudaSetDevice");
    const size_t b = sizeof(float) * (size_t)s->n_params;
    if (set) {
        SCK(cudaMemcpyAsync(s->P[member], set, b, cudaMemcpyHostToDevice, s->stream), "set params");
        int rc = refresh_bf16(s, member);
        if (rc != SBR_OK) return rc;
    }
    if (get) SCK(cudaMemcpyAsync(get, s->P[member], b, cudaMemcpyDeviceToHost, s->stream), "get params");
    SCK(cudaStreamSynchronize(s->stream), "sync");
    return SBR_OK;
}

int sbr_surrogate_fourier(sbr_surrogate* s, int member, float* B)
{
    if (!s || !B || member < 0 || member >= s->opt.n_members) return SBR_ERR_ARG;
    SCK(cudaSetDevice(s->device), "cudaSetDevice");
    SCK(cudaMemcpy(B, s->Bf[member], sizeof(float) * 4 * s->nh, cudaMemcpyDeviceToHost), "get Fourier matrix");
    return SBR_OK;
}

int sbr_surrogate_grads(sbr_surrogate* s, int member, const double* x, const double* y, int64_t n, double* loss,
                        float* grads)
{
    if (!s || !x || !y || n < 128 || n % 128 || member < 0 || member >= s->opt.n_members) return SBR_ERR_ARG;
    SCK(cudaSetDevice(s->device), "cudaSetDevice");
    int rc = ensure_cap(s, (int)n);
    if (rc != SBR_OK) return rc;
    float* x4 = nullptr;
    rc = upload_inputs(s, x, n, &x4);
    if (rc != SBR_OK) return rc;
    std::vector<float> yt((size_t)n * kOut);
    for (size_t i = 0; i < yt.size(); ++i) yt[i] = (float)(y[i] / s->target_scale);
    cudaMemcpyAsync(s->xb, x4, sizeof(float) * kIn * (size_t)n, cudaMemcpyDeviceToDevice, s->stream);
    cudaMemcpyAsync(s->yb, yt.data(), sizeof(float) * yt.size(), cudaMemcpyHostToDevice, s->stream);
    cudaMemsetAsync(s->gerr, 0, sizeof(int), s->stream);
    rc = forward(s, member, (int)n, s->y);
    if (rc == SBR_OK) rc = backward(s, member, (int)n);
    if (rc == SBR_OK) rc = check_gemm_err(s);
    cudaFree(x4);
    if (rc != SBR_OK) return rc;
    double hl = 0.0;
    SCK(cudaMemcpy(&hl, s->loss, sizeof(double), cudaMemcpyDeviceToHost), "copy loss");
    if (loss) *loss = hl / (double)(n * kOut);
    if (grads) SCK(cudaMemcpy(grads, s->G, sizeof(float) * (size_t)s->n_params, cudaMemcpyDeviceToHost), "copy grads");
    return SBR_OK;
}

int sbr_surrogate_train(sbr_surrogate* s, const double* x, const double* y, int64_t n, int epochs, int batch,
                        float lr, float* loss_per_epoch)
{
    if (!s || !x || !y || n < 128 || epochs < 1 || batch < 128 || batch % 128 || !(lr > 0.f)) return SBR_ERR_ARG;
    if (n > (1ll << 31) - 1) return SBR_ERR_ARG;
    SCK(cudaSetDevice(s->device), "cudaSetDevice");
    const int M = (int)std::min<long long>(batch, (n / 128) * 128);
    int rc = ensure_cap(s, M);
    if (rc != SBR_OK) return rc;
    // target scale: RMS of the targets
    double ss = 0.0;
    for (int64_t i = 0; i < n * kOut; ++i) ss += y[i] * y[i];
    s->target_scale = (float)std::max(sqrt(ss / (double)(n * kOut)), 1e-30);
    float *x4 = nullptr, *y4 = nullptr;
    rc = upload_inputs(s, x, n, &x4);
    if (rc != SBR_OK) return rc;
    std::vector<float> yt((size_t)n * kOut);
    for (size_t i = 0; i < yt.size(); ++i) yt[i] = (float)(y[i] / s->target_scale);
    cudaError_t ce = cudaMalloc(&y4, sizeof(float) * yt.size());
    if (ce == cudaSuccess) ce = cudaMemcpy(y4, yt.data(), sizeof(float) * yt.size(), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
        cudaFree(x4);
        SCK(ce, "upload targets");
    }
    const long long steps_per_epoch = n / M;
    // one permutation per epoch on the device; per-epoch squared-error sums on the device
    int* dperm = nullptr;
    double* dloss = nullptr;
    ce = cudaMalloc(&dperm, sizeof(int) * (size_t)n);
    if (ce == cudaSuccess) ce = cudaMalloc(&dloss, sizeof(double) * (size_t)epochs);
    if (ce != cudaSuccess) {
        cudaFree(x4);
        cudaFree(y4);
        cudaFree(dperm);
        SCK(ce, "alloc permutation");
    }
    std::vector<int> perm((size_t)n);
    std::vector<double> hloss((size_t)epochs);
    cudaMemsetAsync(s->gerr, 0, sizeof(int), s->stream);
    const double total_steps = (double)epochs * (double)steps_per_epoch;
    for (int e = 0; e < s->opt.n_members && rc == SBR_OK; ++e) {
        std::mt19937_64 rng(s->opt.seed * 7919 + (uint64_t)e);
        cudaMemsetAsync(dloss, 0, sizeof(double) * (size_t)epochs, s->stream);
        long long call_step = 0;
        for (int ep = 0; ep < epochs && rc == SBR_OK; ++ep) {
            for (int64_t i = 0; i < n; ++i) perm[(size_t)i] = (int)i;
            std::shuffle(perm.begin(), perm.end(), rng);
            // pageable source: the call returns once the host buffer has been consumed
            if (cudaMemcpyAsync(dperm, perm.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, s->stream) !=
                cudaSuccess) {
                rc = sfail(s, SBR_ERR_CUDA, "upload permutation");
                break;
            }
            for (long long st = 0; st < steps_per_epoch && rc == SBR_OK; ++st) {
                k_gather<<<blocks(M, 256), 256, 0, s->stream>>>(x4, y4, dperm + st * M, M, s->xb, s->yb);
                rc = forward(s, e, M, s->y);
                if (rc == SBR_OK) rc = backward(s, e, M, dloss + ep);
                if (rc != SBR_OK) break;
                const long long t = ++s->steps[(size_t)e];
                const float b1 = 0.9f, b2 = 0.999f;
                const float c1 = 1.f / (1.f - powf(b1, (float)t)), c2 = 1.f / (1.f - powf(b2, (float)t));
                // cosine schedule lr -> lr / 100 over this call
                const double ph = (double)(call_step++) / std::max(1.0, total_steps - 1.0);
                const float lr_t = (float)(lr * (0.01 + 0.99 * 0.5 * (1.0 + cos(kPi * ph))));
                k_adam<<<blocks(s->n_params, 256), 256, 0, s->stream>>>(s->P[e], s->Pm[e], s->Pv[e], s->G,
                                                                         s->n_params, lr_t, b1, b2, c1, c2, 1e-8f);
                rc = refresh_bf16(s, e);
            }
        }
        if (rc == SBR_OK &&
            (cudaMemcpyAsync(hloss.data(), dloss, sizeof(double) * (size_t)epochs, cudaMemcpyDeviceToHost,
                             s->stream) != cudaSuccess ||
             cudaStreamSynchronize(s->stream) != cudaSuccess))
            rc = sfail(s, SBR_ERR_CUDA, "copy losses");
        if (rc == SBR_OK && loss_per_epoch)
            for (int ep = 0; ep < epochs; ++ep)
                loss_per_epoch[(size_t)e * epochs + ep] =
                    (float)(hloss[(size_t)ep] / ((double)M * kOut * (double)steps_per_epoch));
    }
    cudaFree(dperm);
    cudaFree(dloss);
    if (rc == SBR_OK) rc = check_gemm_err(s);
    cudaFree(x4);
    cudaFree(y4);
    if (rc == SBR_OK) s->trained = true;
    return rc;
}

int sbr_surrogate_predict(sbr_surrogate* s, const double* x, int64_t n, double* y_mean, float* spread_db)
{
    if (!s || !x || n < 1 || (!y_mean && !spread_db)) return SBR_ERR_ARG;
    if (n > (1ll << 31) - 1) return SBR_ERR_ARG;
    SCK(cudaSetDevice(s->device), "cudaSetDevice");
    // prediction batches of 65536 rows: the GEMMs fill the GPU with two or more tiles per SM
    const int M = (int)std::min<int64_t>(65536, ((n + 127) / 128) * 128);
    int rc = ensure_cap(s, M);
    if (rc != SBR_OK) return rc;
    float* x4 = nullptr;
    rc = upload_inputs(s, x, n, &x4);
    if (rc != SBR_OK) return rc;
    double* dmean = nullptr;
    float* dspread = nullptr;
    cudaError_t ce = cudaMalloc(&dmean, sizeof(double) * kOut * (size_t)n);
    if (ce == cudaSuccess) ce = cudaMalloc(&dspread, sizeof(float) * (size_t)n);
    if (ce != cudaSuccess) {
        cudaFree(x4);
        cudaFree(dmean);
        SCK(ce, "alloc outputs");
    }
    cudaMemsetAsync(s->gerr, 0, sizeof(int), s->stream);
    for (int64_t b0 = 0; b0 < n && rc == SBR_OK; b0 += M) {
        const int cnt = (int)std::min<int64_t>(M, n - b0);
        const int Mp = ((cnt + 127) / 128) * 128;  // padded rows are computed and ignored
        cudaMemsetAsync(s->xb, 0, sizeof(float) * kIn * (size_t)Mp, s->stream);
        cudaMemcpyAsync(s->xb, x4 + kIn * b0, sizeof(float) * kIn * (size_t)cnt, cudaMemcpyDeviceToDevice, s->stream);
        for (int e = 0; e < s->opt.n_members && rc == SBR_OK; ++e)
            rc = forward(s, e, Mp, s->y + (size_t)e * M * kOut, false);
        if (rc == SBR_OK)
            k_ens_stats<<<blocks(cnt, 256), 256, 0, s->stream>>>(s->y, s->opt.n_members, (long long)M * kOut, cnt,
                                                                 s->target_scale, dmean + kOut * b0, dspread + b0);
    }
    if (rc == SBR_OK) rc = check_gemm_err(s);
    if (rc == SBR_OK && y_mean)
        rc = cudaMemcpy(y_mean, dmean, sizeof(double) * kOut * (size_t)n, cudaMemcpyDeviceToHost) == cudaSuccess
                 ? SBR_OK
                 : SBR_ERR_CUDA;
    if (rc == SBR_OK && spread_db)
        rc = cudaMemcpy(spread_db, dspread, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost) == cudaSuccess
                 ? SBR_OK
                 : SBR_ERR_CUDA;
    cudaFree(x4);
    cudaFree(dmean);
    cudaFree(dspread);
    return rc;
}

}  // extern "C"
