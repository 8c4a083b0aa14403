// zk_tc.cuh - 5th-generation tensor-core (tcgen05) pieces for the closure
// network's convolutions: TMEM allocation, shared-memory matrix and
// instruction descriptors, the MMA, its completion through an mbarrier, and
// the TMEM-to-register load. Inline PTX only; sm_100-family (sm_103a) targets.
//
// Operand layout used throughout ("canonical K-major, no swizzle"): an R x K
// FP16 operand is stored as 8 x 8 core matrices (8 rows of 16 bytes, 128
// contiguous bytes each); core matrix (r/8, k/8) starts at
//     (r/8) * SBO + (k/8) * 128 bytes,
// element (r, k) inside it at (r%8)*16 + (k%8)*2 bytes. K-adjacent core
// matrices are contiguous (LBO = 128 B); SBO = (K/8) * 128 B.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>

namespace zk_tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Offset in halves of element (r, k) of a canonical K-major operand with K columns.
__host__ __device__ __forceinline__ int canon_off(int r, int k, int K) {
    return (r >> 3) * (K >> 3) * 64 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

// Shared-memory matrix descriptor: start address, leading (K) and stride (M/N)
// byte offsets in 16-byte units, descriptor version 1 (bit 46), no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, FP16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_f16_f32(int M, int N) {
    return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// TMEM allocation by one full warp: the base address is written to *slot (shared).
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Make generic-proxy shared-memory writes visible to the tensor core (async proxy).
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T, one MMA of shape (M, N, 16); issued by one thread.
__device__ __forceinline__ void mma_f16(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t idesc, int accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive once on the mbarrier when every MMA issued so far by this thread is done.
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait for phase `parity` of the mbarrier with at most `limit` polls; returns
// false if the limit ran out (the caller records the error and moves on).
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t limit) {
    const uint32_t a = smem_u32(mbar);
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred q;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, q;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 32 consecutive FP32 columns of this thread's TMEM lane (warp w reads lanes 32w..32w+31).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------------------
// 3x3 periodic convolution of one 8 x 16 pixel tile as an implicit GEMM:
// D[px][co] = sum_k A[px][k] B[co][k], k = tap * CINP + c, tap = 3 p + q,
// A[px][k] = x16[(py + p - 1) mod H][(px + q - 1) mod W][c] (zero for c >= CIN),
// B[co][k] = W16[co][c][p][q]. M = 128 pixels (TMEM lanes), N = 32 output
// channels (TMEM columns), K = 9 CINP in steps of 16, three taps per A chunk.
// ---------------------------------------------------------------------------
constexpr int kTileH = 8, kTileW = 16, kTilePx = kTileH * kTileW;
constexpr int kCo = 32;
constexpr uint32_t kWaitLimit = 1u << 22;   // mbarrier polls before the block gives up
constexpr uint32_t kSelfTestWaitLimit = 64;  // polls per wait in the self-test of the give-up path

// Taps per A chunk: the im2col tile is built and multiplied three taps at a
// time, so a block needs a third of the A tile in shared memory and more
// blocks fit on an SM (measured 1.5x faster than all nine taps at once).
constexpr int kTaps = 3;

template <int CINP>
constexpr int conv_smem_bytes() { return kTilePx * kTaps * CINP * 2 + kCo * 9 * CINP * 2; }

// IN_F32: input is an FP32 [CIN][H][W] stack (rounded to FP16 here), else NHWC
// FP16 [H][W][CINP]. OUT 0: NHWC FP16 [H][W][32] of tanh(z + bias); OUT 1: the
// network's last 1x1 layer on FP16-rounded tanh(z + bias), FP32 [2][H][W].
// err: set to 1 if the MMA completion was not seen within the poll limit.
template <int CINP, int CIN, bool IN_F32, int OUT>
__global__ void __launch_bounds__(128) conv3_tc_kernel(const void* __restrict__ xin, const __half* __restrict__ wcanon,
                                                       const float* __restrict__ bias, const float* __restrict__ w4,
                                                       const float* __restrict__ b4, void* __restrict__ out, int H,
                                                       int W, int* __restrict__ err, int withhold) {
    constexpr int K = 9 * CINP, KC = kTaps * CINP;          // full K, K of one chunk
    constexpr int ABYTES = kTilePx * KC * 2, BBYTES = kCo * K * 2;
    static_assert(CINP % 16 == 0 && ABYTES % 1024 == 0, "operand tiles must stay 1 KB aligned");
    extern __shared__ __align__(1024) unsigned char smem[];
    __half* As = reinterpret_cast<__half*>(smem);
    __half* Bs = reinterpret_cast<__half*>(smem + ABYTES);
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    const int t = threadIdx.x, warp = t >> 5;
    const int py = blockIdx.y * kTileH + (t >> 4), px = blockIdx.x * kTileW + (t & 15);
    if (warp == 0) tmem_alloc(&tslot, 32);
    if (t == 0) mbar_init(&mbar, 1);
    for (int i = t; i < BBYTES / 16; i += kTilePx)
        reinterpret_cast<uint4*>(Bs)[i] = __ldg(reinterpret_cast<const uint4*>(wcanon) + i);
    bool ok = true;
    uint32_t tbase = 0;
    // withhold != 0 is the self-test of the give-up path: no MMA is issued and nothing is
    // committed, so nothing is in flight and every wait below runs out after a short limit
    const uint32_t limit = withhold ? kSelfTestWaitLimit : kWaitLimit;
#pragma unroll 1
    for (int ch = 0; ch < 9 / kTaps; ++ch) {
        if (ch > 0) {
            // the previous chunk's MMAs read As: they must be done before it is refilled
            ok = mbar_wait(&mbar, (ch - 1) & 1, limit) && ok;
            fence_after_sync();
        }
        // im2col rows of this chunk's taps, all loads in flight together
#pragma unroll
        for (int tj = 0; tj < kTaps; ++tj) {
            const int tap = ch * kTaps + tj;
            int yy = py + tap / 3 - 1, xx = px + tap % 3 - 1;
            yy += yy < 0 ? H : (yy >= H ? -H : 0);
            xx += xx < 0 ? W : (xx >= W ? -W : 0);
            if constexpr (IN_F32) {
                const float* f = reinterpret_cast<const float*>(xin);
                const size_t plane = (size_t)H * W, o = (size_t)yy * W + xx;
                alignas(16) __half hv[CINP];
#pragma unroll
                for (int c = 0; c < CINP; ++c) hv[c] = __float2half_rn(c < CIN ? f[c * plane + o] : 0.f);
#pragma unroll
                for (int c8 = 0; c8 < CINP / 8; ++c8)
                    *reinterpret_cast<uint4*>(As + canon_off(t, tj * CINP + c8 * 8, KC)) = reinterpret_cast<const uint4*>(hv)[c8];
            } else {
                const uint4* src = reinterpret_cast<const uint4*>(reinterpret_cast<const __half*>(xin) + ((size_t)yy * W + xx) * CINP);
#pragma unroll
                for (int c8 = 0; c8 < CINP / 8; ++c8)
                    *reinterpret_cast<uint4*>(As + canon_off(t, tj * CINP + c8 * 8, KC)) = __ldg(src + c8);
            }
        }
        fence_proxy_async();
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
        tbase = tslot;
        if (t == 0 && !withhold) {
            const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
            constexpr uint32_t SBOA = (KC / 8) * 128, SBOB = (K / 8) * 128;
            constexpr uint32_t id = idesc_f16_f32(kTilePx, kCo);
#pragma unroll 1
            for (int s = 0; s < KC / 16; ++s)
                mma_f16(tbase, smem_desc(a0 + 256u * s, 128, SBOA),
                        smem_desc(b0 + 256u * (ch * (KC / 16) + s), 128, SBOB), id, (ch > 0 || s > 0) ? 1 : 0);
            mma_commit(&mbar);
        }
    }
    {
        constexpr int last = 9 / kTaps - 1;
        bool done = mbar_wait(&mbar, last & 1, limit);
        if (!done) done = mbar_wait(&mbar, last & 1, limit);   // in-flight MMAs must finish before TMEM is freed
        ok = ok && done;
    }
    fence_after_sync();
    float acc[32];
    tmem_ld32(tbase + ((uint32_t)(warp * 32) << 16), acc);
    if (!ok && (t & 31) == 0) atomicExch(err, 1);
    if constexpr (OUT == 0) {
        alignas(16) __half hv[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) hv[c] = __float2half_rn(tanhf(acc[c] + bias[c]));
        uint4* o = reinterpret_cast<uint4*>(reinterpret_cast<__half*>(out) + ((size_t)py * W + px) * 32);
#pragma unroll
        for (int c8 = 0; c8 < 4; ++c8) o[c8] = reinterpret_cast<const uint4*>(hv)[c8];
    } else {
        float y0 = b4[0], y1 = b4[1];
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            const float h = __half2float(__float2half_rn(tanhf(acc[c] + bias[c])));
            y0 = fmaf(w4[c], h, y0);
            y1 = fmaf(w4[32 + c], h, y1);
        }
        float* o = reinterpret_cast<float*>(out);
        const size_t i = (size_t)py * W + px;
        o[i] = y0;
        o[(size_t)H * W + i] = y1;
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tbase, 32);
}

}  // namespace zk_tc
