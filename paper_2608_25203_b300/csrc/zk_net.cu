// zk_net.cu - the closure network on the GPU: periodic 3x3 / 1x1 convolutions
// with tanh, its forward and backward passes, the mean-squared-error loss and
// Adam, written as plain CUDA kernels.
//
// Network (fixed shape): x [B][6][H][W] -> conv3x3 6->32, tanh -> conv3x3
// 32->32, tanh -> conv3x3 32->32, tanh -> conv1x1 32->2 -> y [B][2][H][W].
// Convolutions are periodic cross-correlations
//     z[o][i][j] = b[o] + sum_{c,p,q} W[o][c][p][q] h[c][i+p-r][j+q-r]   (mod H, W).
// The weights and the activations entering a convolution are rounded to FP16
// (round to nearest even); products, sums, biases, tanh and every gradient are
// FP32. Backward: dz = dh (1 - h^2) through tanh; dW = sum over pixels of
// dz x shifted input (block partial sums, then a fixed-order reduction, so the
// result is deterministic); dh_in = the convolution of dz with the flipped,
// transposed weights. Adam as published by Kingma & Ba (2015).
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/zk.h"
#include "zk_net_internal.h"
#include "zk_tc.cuh"

namespace {

constexpr int kCin = 6, kWidth = 32, kCout = 2;
constexpr int TS = 16;   // pixel tile edge of every convolution kernel

// parameter layout: W1 b1 W2 b2 W3 b3 W4 b4, weights [out][in][k][k]
__host__ __device__ constexpr int ks_of(int l) { return l == 3 ? 1 : 3; }
__host__ __device__ constexpr int in_of(int l) { return l == 0 ? kCin : kWidth; }
__host__ __device__ constexpr int out_of(int l) { return l == 3 ? kCout : kWidth; }
__host__ __device__ constexpr int wcount(int l) { return out_of(l) * in_of(l) * ks_of(l) * ks_of(l); }
__host__ __device__ constexpr int woff(int l) { return l == 0 ? 0 : woff(l - 1) + wcount(l - 1) + out_of(l - 1); }
__host__ __device__ constexpr int boff(int l) { return woff(l) + wcount(l); }
constexpr int kParams = boff(3) + out_of(3);
static_assert(kParams == 20322, "parameter count of the 6-32-32-32-2 network");

__device__ __forceinline__ float r16(float v) { return __half2float(__float2half_rn(v)); }

enum Epi { EPI_NONE = 0, EPI_TANH = 1, EPI_DTANH = 2 };

// One thread per output pixel, all COUT outputs; a block is a TS x TS tile of
// one sample. Weights as [CIN*KS*KS][COUT] in shared memory (COUT contiguous).
// EPI_DTANH multiplies the result by (1 - aux^2) (the tanh derivative of the
// layer output aux, for the backward pass).
template <int CIN, int COUT, int KS, bool RIN, int EPI>
__global__ void __launch_bounds__(256) conv_fwd_kernel(const float* __restrict__ x, const float* __restrict__ w,
                                                       const float* __restrict__ bias, const float* __restrict__ aux,
                                                       float* __restrict__ y, int H, int W) {
    constexpr int R = KS / 2, TH = TS + 2 * R, KK = KS * KS;
    extern __shared__ __align__(16) float sm[];
    float* sw = sm;
    float* sx = sm + CIN * KK * COUT;
    const size_t plane = (size_t)H * W;
    const size_t b = blockIdx.z;
    x += b * CIN * plane;
    y += b * COUT * plane;
    const int i0 = blockIdx.y * TS - R, j0 = blockIdx.x * TS - R;
    for (int e = threadIdx.x; e < CIN * TH * TH; e += blockDim.x) {
        const int c = e / (TH * TH), rr = e - c * (TH * TH), ii = rr / TH, jj = rr - ii * TH;
        int gi = i0 + ii, gj = j0 + jj;
        gi += gi < 0 ? H : (gi >= H ? -H : 0);
        gj += gj < 0 ? W : (gj >= W ? -W : 0);
        const float v = x[c * plane + (size_t)gi * W + gj];
        sx[e] = RIN ? r16(v) : v;
    }
    for (int e = threadIdx.x; e < COUT * CIN * KK; e += blockDim.x) {
        const int co = e / (CIN * KK), rr = e - co * (CIN * KK);
        sw[rr * COUT + co] = w[e];
    }
    __syncthreads();
    const int ty = threadIdx.x / TS, tx = threadIdx.x % TS;
    float acc[COUT];
#pragma unroll
    for (int co = 0; co < COUT; ++co) acc[co] = bias ? bias[co] : 0.f;
    for (int ci = 0; ci < CIN; ++ci) {
#pragma unroll
        for (int p = 0; p < KS; ++p) {
#pragma unroll
            for (int q = 0; q < KS; ++q) {
                const float v = sx[(ci * TH + ty + p) * TH + tx + q];
                const float* wr = sw + ((ci * KS + p) * KS + q) * COUT;
                if constexpr (COUT % 4 == 0) {
#pragma unroll
                    for (int co = 0; co < COUT; co += 4) {
                        const float4 w4 = *reinterpret_cast<const float4*>(wr + co);
                        acc[co] = fmaf(w4.x, v, acc[co]);
                        acc[co + 1] = fmaf(w4.y, v, acc[co + 1]);
                        acc[co + 2] = fmaf(w4.z, v, acc[co + 2]);
                        acc[co + 3] = fmaf(w4.w, v, acc[co + 3]);
                    }
                } else {
#pragma unroll
                    for (int co = 0; co < COUT; ++co) acc[co] = fmaf(wr[co], v, acc[co]);
                }
            }
        }
    }
    const size_t o = (size_t)(blockIdx.y * TS + ty) * W + blockIdx.x * TS + tx;
#pragma unroll
    for (int co = 0; co < COUT; ++co) {
        float z = acc[co];
        if constexpr (EPI == EPI_TANH) z = tanhf(z);
        if constexpr (EPI == EPI_DTANH) {
            const float h = aux[b * COUT * plane + co * plane + o];
            z *= 1.f - h * h;
        }
        y[co * plane + o] = z;
    }
}

// Weight and bias gradient partial sums of one TS x TS tile of one sample:
// part[block][e] = sum_tile dz[o] * hin16[c] shifted by (p, q), e = ((o*CIN+c)*KS+p)*KS+q;
// part[block][E + o] = sum_tile dz[o].
template <int CIN, int COUT, int KS>
__global__ void __launch_bounds__(256) conv_bwd_w_kernel(const float* __restrict__ dz, const float* __restrict__ hin,
                                                         float* __restrict__ part, int H, int W) {
    constexpr int R = KS / 2, TH = TS + 2 * R, KK = KS * KS, E = COUT * CIN * KK;
    extern __shared__ __align__(16) float sm[];
    float* sdz = sm;                   // [COUT][TS*TS]
    float* sh = sm + COUT * TS * TS;   // [CIN][TH][TH]
    const size_t plane = (size_t)H * W;
    const size_t b = blockIdx.z;
    dz += b * COUT * plane;
    hin += b * CIN * plane;
    const int i0 = blockIdx.y * TS, j0 = blockIdx.x * TS;
    for (int e = threadIdx.x; e < COUT * TS * TS; e += blockDim.x) {
        const int c = e / (TS * TS), rr = e - c * (TS * TS), ii = rr / TS, jj = rr - ii * TS;
        sdz[e] = dz[c * plane + (size_t)(i0 + ii) * W + j0 + jj];
    }
    for (int e = threadIdx.x; e < CIN * TH * TH; e += blockDim.x) {
        const int c = e / (TH * TH), rr = e - c * (TH * TH), ii = rr / TH, jj = rr - ii * TH;
        int gi = i0 - R + ii, gj = j0 - R + jj;
        gi += gi < 0 ? H : (gi >= H ? -H : 0);
        gj += gj < 0 ? W : (gj >= W ? -W : 0);
        sh[e] = r16(hin[c * plane + (size_t)gi * W + gj]);
    }
    __syncthreads();
    const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    float* out = part + blk * (E + COUT);
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const int co = e / (CIN * KK), rr = e - co * (CIN * KK), ci = rr / KK, pq = rr - ci * KK;
        const int p = pq / KS, q = pq - p * KS;
        const float* d = sdz + co * TS * TS;
        const float* hh = sh + ci * TH * TH + p * TH + q;
        float acc = 0.f;
        for (int ty = 0; ty < TS; ++ty) {
#pragma unroll
            for (int tx = 0; tx < TS; ++tx) acc = fmaf(d[ty * TS + tx], hh[ty * TH + tx], acc);
        }
        out[e] = acc;
    }
    for (int co = threadIdx.x; co < COUT; co += blockDim.x) {
        float s = 0.f;
        for (int k = 0; k < TS * TS; ++k) s += sdz[co * TS * TS + k];
        out[E + co] = s;
    }
}

// out[e] = sum over blocks k (in order) of part[k * stride + e], FP64 sum.
__global__ void reduce_parts_kernel(const float* __restrict__ part, int nblk, int stride, float* __restrict__ out, int n) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    double s = 0.0;
    for (int k = 0; k < nblk; ++k) s += (double)part[(size_t)k * stride + e];
    out[e] = (float)s;
}

// d = y - t; dy = scale * d; per-block FP64 sums of d^2 into part[blockIdx.x].
__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ dy,
                           double* __restrict__ part, size_t n, float scale) {
    double s = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        dy[i] = scale * d;
        s += (double)d * (double)d;
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red[w];
        part[blockIdx.x] = a;
    }
}

// Data preparation of the closure's training set ([n][c][hw] FP32, channel-major per sample):
// sums of squares per channel, block (channel ch, slice b) over elements i = b, b + nb, ... of
// the channel's n*hw values, reduced in a fixed order (deterministic), FP64 accumulation.
__global__ void __launch_bounds__(256) chan_sumsq_kernel(const float* __restrict__ x, long long n, int c, int hw,
                                                         int nb, double* __restrict__ part) {
    const int ch = blockIdx.y;
    const long long per = n * hw;
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < per; i += (long long)nb * blockDim.x) {
        const long long smp = i / hw, off = i - smp * hw;
        const double v = x[(smp * c + ch) * hw + off];
        acc += v * v;
    }
    __shared__ double red[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[(long long)ch * nb + blockIdx.x] = t;
    }
}

// rms[ch] = sqrt(sum of the channel's partials / count), the partials taken in order.
__global__ void chan_rms_kernel(const double* __restrict__ part, int c, int nb, double count, float* __restrict__ rms) {
    const int ch = blockIdx.x * blockDim.x + threadIdx.x;
    if (ch >= c) return;
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += part[(long long)ch * nb + b];
    rms[ch] = (float)sqrt(t / count);
}

// x[smp][ch][:] *= mul[ch] in place.
__global__ void chan_scale_kernel(float* __restrict__ x, long long total, int c, int hw, const float* __restrict__ mul) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)((i / hw) % c);
        x[i] *= mul[ch];
    }
}

__global__ void sum_kernel(const double* __restrict__ part, int n, double scale, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += part[i];
        *out = s * scale;
    }
}

__global__ void adam_kernel(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mm = b1 * m[i] + (1.f - b1) * gi;
    const float vv = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mm;
    v[i] = vv;
    th[i] -= lr * (mm * c1) / (sqrtf(vv * c2) + eps);
}

// FP16-rounded copy of the weights (biases copied as they are), and for each
// layer the flipped, transposed weights Wf[c][o][p][q] = W16[o][c][K-1-p][K-1-q].
__global__ void prep_weights_kernel(const float* __restrict__ th, float* __restrict__ w16, float* __restrict__ wf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    int l = 0;
    while (l < 3 && i >= woff(l + 1)) ++l;
    const int e = i - woff(l);
    if (e >= wcount(l)) { w16[i] = th[i]; wf[i] = 0.f; return; }   // bias
    const int K = ks_of(l), KK = K * K, CI = in_of(l);
    const float v = r16(th[i]);
    w16[i] = v;
    const int o = e / (CI * KK), rr = e - o * (CI * KK), c = rr / KK, pq = rr - c * KK, p = pq / K, q = pq - p * K;
    wf[woff(l) + ((c * out_of(l) + o) * K + (K - 1 - p)) * K + (K - 1 - q)] = v;
}

// Tensor-core inference: the three 3x3 layers' FP16-rounded weights as the B
// operands of zk_tc::conv3_tc_kernel (canonical K-major, k = tap * CINP + c,
// zero for the padded input channels c >= CIN): layer 1 [32][144], layers 2-3 [32][288].
constexpr int kTcK1 = 9 * 16, kTcK2 = 9 * 32;
constexpr int kTcOff2 = kWidth * kTcK1, kTcOff3 = kTcOff2 + kWidth * kTcK2, kTcTotal = kTcOff3 + kWidth * kTcK2;

__global__ void prep_canon_kernel(const float* __restrict__ th, __half* __restrict__ wc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kTcTotal) return;
    const int l = i < kTcOff2 ? 0 : (i < kTcOff3 ? 1 : 2);
    const int e = i - (l == 0 ? 0 : (l == 1 ? kTcOff2 : kTcOff3));
    const int K = l == 0 ? kTcK1 : kTcK2, CINP = K / 9, CI = in_of(l);
    const int co = e / K, k = e - co * K, tap = k / CINP, c = k - tap * CINP;
    const float v = c < CI ? r16(th[woff(l) + ((co * CI + c) * 3 + tap / 3) * 3 + tap % 3]) : 0.f;
    wc[(i - e) + zk_tc::canon_off(co, k, K)] = __float2half_rn(v);
}

template <int CIN, int COUT, int KS, bool RIN, int EPI>
cudaError_t conv_fwd(const float* x, const float* w, const float* bias, const float* aux, float* y, int B, int H,
                     int W, cudaStream_t s) {
    constexpr int TH = TS + 2 * (KS / 2);
    const size_t smem = (size_t)(CIN * KS * KS * COUT + CIN * TH * TH) * sizeof(float);
    auto fn = conv_fwd_kernel<CIN, COUT, KS, RIN, EPI>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    fn<<<dim3(W / TS, H / TS, B), 256, smem, s>>>(x, w, bias, aux, y, H, W);
    return cudaGetLastError();
}

template <int CIN, int COUT, int KS>
cudaError_t conv_bwd_w(const float* dz, const float* hin, float* part, float* out, int B, int H, int W, cudaStream_t s) {
    constexpr int TH = TS + 2 * (KS / 2), E = COUT * CIN * KS * KS;
    const size_t smem = (size_t)(COUT * TS * TS + CIN * TH * TH) * sizeof(float);
    auto fn = conv_bwd_w_kernel<CIN, COUT, KS>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const dim3 grid(W / TS, H / TS, B);
    fn<<<grid, 256, smem, s>>>(dz, hin, part, H, W);
    const int nblk = (int)(grid.x * grid.y * grid.z);
    reduce_parts_kernel<<<(E + COUT + 255) / 256, 256, 0, s>>>(part, nblk, E + COUT, out, E + COUT);
    return cudaGetLastError();
}

}  // namespace

struct zk_net {
    float* theta = nullptr;   // FP32 master parameters
    float* m = nullptr;
    float* v = nullptr;
    float* grad = nullptr;
    float* w16 = nullptr;     // FP16-rounded weights (+ biases), theta layout
    float* wf = nullptr;      // flipped / transposed weights, theta layout
    int t = 0;                // Adam steps taken
    bool prepared = false;
    size_t cap = 0;           // pixels the activation buffers hold
    float *h1 = nullptr, *h2 = nullptr, *h3 = nullptr, *y = nullptr, *ga = nullptr, *gb = nullptr;
    float* part = nullptr;
    size_t part_cap = 0;
    double* dpart = nullptr;  // loss partials [1024] + loss [1]
    const float* x = nullptr; // input of the last forward pass (caller memory)
    int B = 0, H = 0, W = 0;
    int infer_mode = 1;       // inference on 0 = the FP32 SIMT kernels, 1 = tensor cores (default),
                              // 2 = tensor-core self-test with the MMAs withheld
    __half* wc = nullptr;     // canonical FP16 B operands of the tensor-core layers
    __half *a16 = nullptr, *b16 = nullptr;   // NHWC FP16 activations [H][W][32] (inference)
    int* err = nullptr;       // set by a tensor-core block whose MMA wait ran out
    std::vector<void*> bufs;  // activation-sized allocations (freed on growth)
};

namespace {

zk_status net_alloc(void** p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) { *p = nullptr; cudaGetLastError(); return ZK_ENOMEM; }
    if (cudaMemset(*p, 0, bytes) != cudaSuccess) return ZK_ECUDA;
    return ZK_OK;
}

void free_bufs(zk_net* n) {
    for (void* p : n->bufs) cudaFree(p);
    n->bufs.clear();
    n->h1 = n->h2 = n->h3 = n->y = n->ga = n->gb = nullptr;
    n->a16 = n->b16 = nullptr;
    n->part = nullptr;
    n->cap = 0;
    n->part_cap = 0;
}

bool shape_ok(int B, int H, int W) { return B >= 1 && H >= TS && W >= TS && H % TS == 0 && W % TS == 0; }

cudaError_t prepare(zk_net* n, cudaStream_t s) {
    if (n->prepared) return cudaSuccess;
    prep_weights_kernel<<<(kParams + 255) / 256, 256, 0, s>>>(n->theta, n->w16, n->wf);
    prep_canon_kernel<<<(kTcTotal + 255) / 256, 256, 0, s>>>(n->theta, n->wc);
    n->prepared = true;
    return cudaGetLastError();
}

template <int CINP, int CIN, bool IN_F32, int OUT>
cudaError_t tc_layer(const void* x, const __half* wc, const float* bias, const float* w4, const float* b4, void* out,
                     int H, int W, int* err, int withhold, cudaStream_t s) {
    constexpr int smem = zk_tc::conv_smem_bytes<CINP>();
    auto fn = zk_tc::conv3_tc_kernel<CINP, CIN, IN_F32, OUT>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    fn<<<dim3(W / zk_tc::kTileW, H / zk_tc::kTileH), zk_tc::kTilePx, smem, s>>>(x, wc, bias, w4, b4, out, H, W, err,
                                                                                 withhold);
    return cudaGetLastError();
}

// Inference of one sample on the tensor cores: layer 1 from the FP32 features,
// layers 2 and 3 through NHWC FP16 activations, layer 4 in layer 3's epilogue.
cudaError_t tc_forward(zk_net* n, const float* x, int H, int W, cudaStream_t s) {
    cudaError_t e = prepare(n, s);
    const float* th = n->theta;
    const int wh = n->infer_mode == 2 ? 1 : 0;
    if (e == cudaSuccess)
        e = tc_layer<16, kCin, true, 0>(x, n->wc, th + boff(0), nullptr, nullptr, n->a16, H, W, n->err, wh, s);
    if (e == cudaSuccess)
        e = tc_layer<32, kWidth, false, 0>(n->a16, n->wc + kTcOff2, th + boff(1), nullptr, nullptr, n->b16, H, W, n->err,
                                           wh, s);
    if (e == cudaSuccess)
        e = tc_layer<32, kWidth, false, 1>(n->b16, n->wc + kTcOff3, th + boff(2), n->w16 + woff(3), th + boff(3), n->y,
                                           H, W, n->err, wh, s);
    return e;
}

cudaError_t forward(zk_net* n, const float* x, int B, int H, int W, cudaStream_t s) {
    cudaError_t e = prepare(n, s);
    const float* w = n->w16;
    const float* th = n->theta;
    if (e == cudaSuccess)
        e = conv_fwd<kCin, kWidth, 3, true, EPI_TANH>(x, w + woff(0), th + boff(0), nullptr, n->h1, B, H, W, s);
    if (e == cudaSuccess)
        e = conv_fwd<kWidth, kWidth, 3, true, EPI_TANH>(n->h1, w + woff(1), th + boff(1), nullptr, n->h2, B, H, W, s);
    if (e == cudaSuccess)
        e = conv_fwd<kWidth, kWidth, 3, true, EPI_TANH>(n->h2, w + woff(2), th + boff(2), nullptr, n->h3, B, H, W, s);
    if (e == cudaSuccess)
        e = conv_fwd<kWidth, kCout, 1, true, EPI_NONE>(n->h3, w + woff(3), th + boff(3), nullptr, n->y, B, H, W, s);
    return e;
}

// dL/dtheta into n->grad from dL/dy (dy: [B][2][H][W]); dx optional.
cudaError_t backward(zk_net* n, const float* dy, float* dx, cudaStream_t s) {
    const int B = n->B, H = n->H, W = n->W;
    const float* wf = n->wf;
    float* g = n->grad;
    cudaError_t e = conv_bwd_w<kWidth, kCout, 1>(dy, n->h3, n->part, g + woff(3), B, H, W, s);
    // dz3 = (W4f * dy) (1 - h3^2)
    if (e == cudaSuccess) e = conv_fwd<kCout, kWidth, 1, false, EPI_DTANH>(dy, wf + woff(3), nullptr, n->h3, n->ga, B, H, W, s);
    if (e == cudaSuccess) e = conv_bwd_w<kWidth, kWidth, 3>(n->ga, n->h2, n->part, g + woff(2), B, H, W, s);
    if (e == cudaSuccess) e = conv_fwd<kWidth, kWidth, 3, false, EPI_DTANH>(n->ga, wf + woff(2), nullptr, n->h2, n->gb, B, H, W, s);
    if (e == cudaSuccess) e = conv_bwd_w<kWidth, kWidth, 3>(n->gb, n->h1, n->part, g + woff(1), B, H, W, s);
    if (e == cudaSuccess) e = conv_fwd<kWidth, kWidth, 3, false, EPI_DTANH>(n->gb, wf + woff(1), nullptr, n->h1, n->ga, B, H, W, s);
    if (e == cudaSuccess) e = conv_bwd_w<kCin, kWidth, 3>(n->ga, n->x, n->part, g + woff(0), B, H, W, s);
    if (e == cudaSuccess && dx) e = conv_fwd<kWidth, kCin, 3, false, EPI_NONE>(n->ga, wf + woff(0), nullptr, nullptr, dx, B, H, W, s);
    return e;
}

}  // namespace

zk_status zk_net_reserve(zk_net* n, size_t pixels) {
    if (!n || pixels == 0) return ZK_EINVAL;
    if (pixels <= n->cap) return ZK_OK;
    free_bufs(n);
    float** act[6] = {&n->h1, &n->h2, &n->h3, &n->ga, &n->gb, &n->y};
    const size_t ch[6] = {kWidth, kWidth, kWidth, kWidth, kWidth, kCout};
    for (int i = 0; i < 6; ++i) {
        void* p = nullptr;
        zk_status st = net_alloc(&p, pixels * ch[i] * sizeof(float));
        if (st != ZK_OK) { free_bufs(n); return st; }
        n->bufs.push_back(p);
        *act[i] = (float*)p;
    }
    for (__half** q : {&n->a16, &n->b16}) {
        void* p = nullptr;
        zk_status st = net_alloc(&p, pixels * kWidth * sizeof(__half));
        if (st != ZK_OK) { free_bufs(n); return st; }
        n->bufs.push_back(p);
        *q = (__half*)p;
    }
    // weight-gradient partials: one row per 16 x 16 tile of the largest layer
    const size_t rows = pixels / (TS * TS) + 1;
    const size_t per = (size_t)kWidth * kWidth * 9 + kWidth;
    void* p = nullptr;
    zk_status st = net_alloc(&p, rows * per * sizeof(float));
    if (st != ZK_OK) { free_bufs(n); return st; }
    n->bufs.push_back(p);
    n->part = (float*)p;
    n->part_cap = rows * per;
    n->cap = pixels;
    return ZK_OK;
}

cudaError_t zk_net_infer(zk_net* n, const float* x, const float** y, int B, int H, int W, cudaStream_t s) {
    if (!n || !y || !shape_ok(B, H, W) || (size_t)B * H * W > n->cap) return cudaErrorInvalidValue;
    *y = n->y;
    if (n->infer_mode >= 1 && B == 1) return tc_forward(n, x, H, W, s);
    return forward(n, x, B, H, W, s);
}

extern "C" {

zk_status zk_net_channel_rms(const float* x, long long n, int c, int hw, float* rms, void* stream) {
    if (!x || !rms || n <= 0 || c <= 0 || c > 64 || hw <= 0) return ZK_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    constexpr int kSlices = 256;
    double* part = nullptr;
    float* drms = nullptr;
    if (cudaMallocAsync((void**)&part, sizeof(double) * kSlices * c, s) != cudaSuccess) { cudaGetLastError(); return ZK_ENOMEM; }
    if (cudaMallocAsync((void**)&drms, sizeof(float) * c, s) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeAsync(part, s);
        return ZK_ENOMEM;
    }
    chan_sumsq_kernel<<<dim3(kSlices, c), 256, 0, s>>>(x, n, c, hw, kSlices, part);
    chan_rms_kernel<<<1, 64, 0, s>>>(part, c, kSlices, (double)n * hw, drms);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(rms, drms, sizeof(float) * c, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(part, s);
    cudaFreeAsync(drms, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? ZK_OK : ZK_ECUDA;
}

zk_status zk_net_scale_channels(float* x, long long n, int c, int hw, const float* mul, void* stream) {
    if (!x || !mul || n <= 0 || c <= 0 || c > 64 || hw <= 0) return ZK_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    float* dmul = nullptr;
    if (cudaMallocAsync((void**)&dmul, sizeof(float) * c, s) != cudaSuccess) { cudaGetLastError(); return ZK_ENOMEM; }
    cudaError_t e = cudaMemcpyAsync(dmul, mul, sizeof(float) * c, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        const long long total = n * c * (long long)hw;
        const int blocks = (int)std::min<long long>((total + 255) / 256, 148LL * 32);
        chan_scale_kernel<<<blocks, 256, 0, s>>>(x, total, c, hw, dmul);
        e = cudaGetLastError();
    }
    cudaFreeAsync(dmul, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? ZK_OK : ZK_ECUDA;
}

void zk_net_destroy(zk_net* n) {
    if (!n) return;
    free_bufs(n);
    void* p[9] = {n->theta, n->m, n->v, n->grad, n->w16, n->wf, n->dpart, n->wc, n->err};
    for (void* q : p) if (q) cudaFree(q);
    delete n;
}

zk_status zk_net_create(zk_net** out, int cin, int width, int cout) {
    if (!out) return ZK_EINVAL;
    *out = nullptr;
    if (cin != kCin || width != kWidth || cout != kCout) return ZK_EUNSUPPORTED;
    zk_net* n = new (std::nothrow) zk_net();
    if (!n) return ZK_ENOMEM;
    zk_status st = ZK_OK;
    float** p[6] = {&n->theta, &n->m, &n->v, &n->grad, &n->w16, &n->wf};
    for (int i = 0; i < 6 && st == ZK_OK; ++i) {
        void* q = nullptr;
        st = net_alloc(&q, kParams * sizeof(float));
        *p[i] = (float*)q;
    }
    if (st == ZK_OK) {
        void* q = nullptr;
        st = net_alloc(&q, 1025 * sizeof(double));
        n->dpart = (double*)q;
    }
    if (st == ZK_OK) {
        void* q = nullptr;
        st = net_alloc(&q, kTcTotal * sizeof(__half));
        n->wc = (__half*)q;
    }
    if (st == ZK_OK) {
        void* q = nullptr;
        st = net_alloc(&q, sizeof(int));
        n->err = (int*)q;
    }
    if (st != ZK_OK) { zk_net_destroy(n); return st; }
    *out = n;
    return ZK_OK;
}

zk_status zk_net_set_inference(zk_net* n, int mode) {
    if (!n || mode < 0 || mode > 2) return ZK_EINVAL;
    n->infer_mode = mode;
    return ZK_OK;
}

zk_status zk_net_predict(zk_net* n, const float* x, float* y, int nz, int nx, void* stream) {
    if (!n || !x || !y || !shape_ok(1, nz, nx)) return ZK_EINVAL;
    zk_status st = zk_net_reserve(n, (size_t)nz * nx);
    if (st != ZK_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const float* out = nullptr;
    if (cudaMemsetAsync(n->err, 0, sizeof(int), s) != cudaSuccess) return ZK_ECUDA;
    cudaError_t e = zk_net_infer(n, x, &out, 1, nz, nx, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(y, out, (size_t)kCout * nz * nx * sizeof(float), cudaMemcpyDeviceToDevice, s);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, n->err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return ZK_ECUDA;
    return herr ? ZK_ETIMEOUT : ZK_OK;
}

zk_status zk_net_param_count(const zk_net* n, int* count) {
    if (!n || !count) return ZK_EINVAL;
    *count = kParams;
    return ZK_OK;
}

zk_status zk_net_set_params(zk_net* n, const float* theta, int on_device) {
    if (!n || !theta) return ZK_EINVAL;
    const size_t b = kParams * sizeof(float);
    if (cudaMemcpy(n->theta, theta, b, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice) != cudaSuccess)
        return ZK_ECUDA;
    if (cudaMemset(n->m, 0, b) != cudaSuccess || cudaMemset(n->v, 0, b) != cudaSuccess) return ZK_ECUDA;
    n->t = 0;
    n->prepared = false;
    return ZK_OK;
}

zk_status zk_net_get_params(zk_net* n, float* theta, int on_device) {
    if (!n || !theta) return ZK_EINVAL;
    if (cudaMemcpy(theta, n->theta, kParams * sizeof(float), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost) !=
        cudaSuccess)
        return ZK_ECUDA;
    return ZK_OK;
}

zk_status zk_net_forward(zk_net* n, const float* x, float* y, int batch, int nz, int nx, void* stream) {
    if (!n || !x || !shape_ok(batch, nz, nx)) return ZK_EINVAL;
    zk_status st = zk_net_reserve(n, (size_t)batch * nz * nx);
    if (st != ZK_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = forward(n, x, batch, nz, nx, s);
    n->x = x; n->B = batch; n->H = nz; n->W = nx;
    if (e == cudaSuccess && y)
        e = cudaMemcpyAsync(y, n->y, (size_t)batch * kCout * nz * nx * sizeof(float), cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? ZK_OK : ZK_ECUDA;
}

zk_status zk_net_backward(zk_net* n, const float* dy, float* grad, float* dx, void* stream) {
    if (!n || !dy) return ZK_EINVAL;
    if (!n->x) return ZK_ESTATE;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = backward(n, dy, dx, s);
    if (e == cudaSuccess && grad) e = cudaMemcpyAsync(grad, n->grad, kParams * sizeof(float), cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? ZK_OK : ZK_ECUDA;
}

zk_status zk_net_adam(zk_net* n, const float* grad, double lr, void* stream) {
    if (!n || !(lr >= 0)) return ZK_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const float* g = grad ? grad : n->grad;
    n->t += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 / (1.0 - std::pow(b1, n->t))), c2 = (float)(1.0 / (1.0 - std::pow(b2, n->t)));
    adam_kernel<<<(kParams + 255) / 256, 256, 0, s>>>(n->theta, g, n->m, n->v, kParams, (float)lr, (float)b1, (float)b2,
                                                      1e-8f, c1, c2);
    n->prepared = false;
    return cudaGetLastError() == cudaSuccess ? ZK_OK : ZK_ECUDA;
}

zk_status zk_net_train_step(zk_net* n, const float* x, const float* target, int batch, int nz, int nx, double lr,
                            double* loss, void* stream) {
    if (!n || !x || !target || !shape_ok(batch, nz, nx) || !(lr >= 0)) return ZK_EINVAL;
    zk_status st = zk_net_forward(n, x, nullptr, batch, nz, nx, stream);
    if (st != ZK_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t cnt = (size_t)batch * kCout * nz * nx;
    const int blocks = 1024;
    // dL/dy into gb's first 2 channels' worth of storage (gb holds 32 channels)
    float* dy = n->gb;
    mse_kernel<<<blocks, 256, 0, s>>>(n->y, target, dy, n->dpart, cnt, (float)(2.0 / (double)cnt));
    sum_kernel<<<1, 32, 0, s>>>(n->dpart, blocks, 1.0 / (double)cnt, n->dpart + 1024);
    if (cudaGetLastError() != cudaSuccess) return ZK_ECUDA;
    // backward uses ga/gb as scratch: move dy to the output buffer first
    if (cudaMemcpyAsync(n->y, dy, cnt * sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess) return ZK_ECUDA;
    if (backward(n, n->y, nullptr, s) != cudaSuccess) return ZK_ECUDA;
    st = zk_net_adam(n, nullptr, lr, stream);
    if (st != ZK_OK) return st;
    if (loss) {
        if (cudaMemcpyAsync(loss, n->dpart + 1024, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return ZK_ECUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return ZK_ECUDA;
    }
    return ZK_OK;
}

}  // extern "C"
