// zk_dftmma.cuh - split-precision DFT-GEMM stage for the padded line FFTs.
//
// The precision form of the right-hand side runs the innermost radix-8 stage
// of the default long-line plans (block 8, stride 1: a length-8 DFT of 8
// contiguous complex values, no twiddles, in both the DIF and the DIT
// direction) as a matrix product on the tensor cores. With F = Fr + i Fi the
// length-8 DFT matrix and the 8 blocks of a group as the columns of X:
//     [Re Y]   [Fr  -Fi] [Re X]
//     [Im Y] = [Fi   Fr] [Im X],
// one real 16 x 16 x 8 product (mma.sync m16n8k16, FP32 accumulation) per
// group of 8 blocks. Each FP32 operand v is split into a 16-bit high part
// h = rn(v) and low part l = rn(v - h), and the product takes the three terms
// h h' + h l' + l h'. With u the unit roundoff of the 16-bit format (2^-11 for
// FP16, 2^-8 for BF16), the dropped l l' term and the rounding of l are each at
// most u^2 of the operands: 2^-22 for FP16 parts, 2^-16 for BF16 parts (less on
// average). Two forms:
//   SPLIT_BF16: BF16 parts (FP32 exponent range, 8-bit significands);
//   SPLIT_FP16: FP16 parts (11-bit significands). Every block (a GEMM column)
//     is first scaled by a power of two that puts its largest component in
//     [2^13, 2^14), which keeps the FP16 parts finite; the outputs are scaled
//     back exactly.
// mma.sync fragment layout of m16n8k16 (PTX ISA): lane = 4 * gid + t;
//   A (16 x 16, row major): regs {A[gid][2t..2t+1], A[gid+8][2t..2t+1],
//                                 A[gid][2t+8..2t+9], A[gid+8][2t+8..2t+9]};
//   B (16 x 8, column major): regs {B[2t..2t+1][gid], B[2t+8..2t+9][gid]};
//   C/D (16 x 8, FP32): {D[gid][2t], D[gid][2t+1], D[gid+8][2t], D[gid+8][2t+1]}.
// So lane (gid, t) loads elements 2t, 2t+1 of block gid and stores element
// gid of blocks 2t and 2t+1.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "zk_fft2.cuh"

namespace zk {

enum { SPLIT_BF16 = 2, SPLIT_FP16 = 3 };   // plan variants V that use the DFT-GEMM stage

// cos and sin of 2 pi q / 16 (q taken mod 16) from the first-quadrant values.
__device__ __forceinline__ float2 cs16(int q) {
    const float c1 = 0.923879532511286756f, c2 = 0.707106781186547524f, c3 = 0.382683432365089772f;
    q &= 15;
    const int m = q & 3, quad = q >> 2;
    const float a = m == 0 ? 1.f : m == 1 ? c1 : m == 2 ? c2 : c3;   // cos(m * 2 pi / 16)
    const float b = m == 0 ? 0.f : m == 1 ? c3 : m == 2 ? c2 : c1;   // sin(m * 2 pi / 16)
    // quadrant rotation by quad * 90 degrees: (c, s) -> (-s, c)
    const float c = quad == 0 ? a : quad == 1 ? -b : quad == 2 ? -a : b;
    const float s = quad == 0 ? b : quad == 1 ? a : quad == 2 ? -b : -a;
    return make_float2(c, s);
}

template <int PREC> struct Split;
template <> struct Split<SPLIT_BF16> {
    // packed high parts of (a, b) (a in the low half) and the packed low parts
    static __device__ __forceinline__ void run(float a, float b, uint32_t& hi, uint32_t& lo) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    }
};
template <> struct Split<SPLIT_FP16> {
    static __device__ __forceinline__ void run(float a, float b, uint32_t& hi, uint32_t& lo) {
        const __half2 h = __floats2half2_rn(a, b);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    }
};

template <int PREC>
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    if constexpr (PREC == SPLIT_BF16) {
        asm(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    } else {
        asm(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
}

// This lane's A fragments of [[Fr, -Fi], [Fi, Fr]] (high and low parts) for direction INV.
template <bool INV, int PREC>
struct DftFrags {
    uint32_t hi[4], lo[4];
    __device__ __forceinline__ DftFrags(int lane) {
        const int gid = lane >> 2, t = lane & 3;
        // F[r][c] = exp(-+ 2 pi i r c / 8) = cos - + i sin of 2 pi (2 r c) / 16
        const float sg = INV ? 1.f : -1.f;
        const float2 e0 = cs16(2 * gid * (2 * t)), e1 = cs16(2 * gid * (2 * t + 1));
        const float fr0 = e0.x, fr1 = e1.x, fi0 = sg * e0.y, fi1 = sg * e1.y;
        Split<PREC>::run(fr0, fr1, hi[0], lo[0]);     // rows gid (Re Y), cols 2t.. (Re X): Fr
        Split<PREC>::run(fi0, fi1, hi[1], lo[1]);     // rows gid + 8 (Im Y), cols 2t.. (Re X): Fi
        Split<PREC>::run(-fi0, -fi1, hi[2], lo[2]);   // rows gid (Re Y), cols 2t + 8.. (Im X): -Fi
        Split<PREC>::run(fr0, fr1, hi[3], lo[3]);     // rows gid + 8 (Im Y), cols 2t + 8.. (Im X): Fr
    }
};

// Slot of block b of the block-8 stage in the padded line layout (element e at
// slot + e): stage_pbase of that stage.
__device__ __forceinline__ int blk8_slot(int b) { return 8 * b + (b >> 1); }

// One group of 8 blocks transformed in place by one warp. Loads finish before
// stores (__syncwarp), so the group may be overwritten by its own results.
template <bool INV, int PREC>
__device__ __forceinline__ void dft8_group(float2* line, int grp, int lane, const DftFrags<INV, PREC>& F) {
    const int gid = lane >> 2, t = lane & 3;
    const float2* in = line + blk8_slot(8 * grp + gid);
    float2 x0 = in[2 * t], x1 = in[2 * t + 1];
    float inv0 = 1.f, inv1 = 1.f;
    if constexpr (PREC == SPLIT_FP16) {
        // power-of-two scale of this lane's input block: largest component in [2^13, 2^14)
        float m = fmaxf(fmaxf(fabsf(x0.x), fabsf(x0.y)), fmaxf(fabsf(x1.x), fabsf(x1.y)));
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
        const int e = (int)((__float_as_uint(m) >> 23) & 0xffu);
        const int se = min(max(267 - e, 1), 253);
        const float sc = __uint_as_float((uint32_t)se << 23);
        const float isc = __uint_as_float((uint32_t)(254 - se) << 23);
        x0.x *= sc; x0.y *= sc; x1.x *= sc; x1.y *= sc;
        // this lane's outputs belong to blocks 2t and 2t + 1, whose inputs lanes 8t and 8t + 4 hold
        inv0 = __shfl_sync(0xffffffffu, isc, 8 * t);
        inv1 = __shfl_sync(0xffffffffu, isc, 8 * t + 4);
    }
    __syncwarp();
    uint32_t rh, rl, ih, il;
    Split<PREC>::run(x0.x, x1.x, rh, rl);
    Split<PREC>::run(x0.y, x1.y, ih, il);
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    // small terms first: A_lo X_hi, A_hi X_lo, then A_hi X_hi
    mma16816<PREC>(d, F.lo, rh, ih);
    mma16816<PREC>(d, F.hi, rl, il);
    mma16816<PREC>(d, F.hi, rh, ih);
    line[blk8_slot(8 * grp + 2 * t) + gid] = make_float2(d[0] * inv0, d[2] * inv0);
    line[blk8_slot(8 * grp + 2 * t + 1) + gid] = make_float2(d[1] * inv1, d[3] * inv1);
}

// The stage over one line by its line group (TL a multiple of 32: whole warps).
template <int N, int TL, bool INV, int PREC>
__device__ __forceinline__ void dft8_line(float2* line, int lt) {
    static_assert(TL % 32 == 0 && N % 64 == 0, "DFT-GEMM stage needs whole warps and 8-block groups");
    const int lane = lt & 31;
    const DftFrags<INV, PREC> F(lane);
    for (int grp = lt >> 5; grp < N / 64; grp += TL / 32) dft8_group<INV, PREC>(line, grp, lane, F);
}

// The stage over one line by the whole block (nt threads, a multiple of 32).
template <int N, bool INV, int PREC>
__device__ __forceinline__ void dft8_line_blk(float2* line, int tid, int nt) {
    const int lane = tid & 31;
    const DftFrags<INV, PREC> F(lane);
    for (int grp = tid >> 5; grp < N / 64; grp += nt >> 5) dft8_group<INV, PREC>(line, grp, lane, F);
}

// The swizzled thread order of the 8-wide radix-8 stage (zk_fft2.cuh) in these plans: taken
// for 3072-point lines; at 1536 points it raised ptxas's register count of the row kernel
// from 64 to 100, which cost more than the bank conflict it removes.
template <int N> constexpr bool kSplitSwz = N >= 3072;

// Plans with the DFT-GEMM stage: the radices (R1, 8, 8, 8), line-group width
// and twiddle table of the default (V = 0) plan of the same length; only the
// block-8 stage is replaced.
template <int N, int PREC>
struct IPlanSplit {
    using B0 = IPlan<N, 0>;
    static constexpr int TL = B0::TL, R1 = B0::R1, NSTAGE = B0::NSTAGE;
    static_assert(NSTAGE == 4 && B0::RADICES[1] == 8 && B0::RADICES[2] == 8 && B0::RADICES[3] == 8,
                  "split-precision plans replace the last radix-8 stage of an (R1, 8, 8, 8) plan");
    static constexpr int OFF = (R1 - 1) * (N / R1);   // table offset of the block-N/R1 stage
    template <bool INV, typename T, class Load>
    static __device__ __forceinline__ void dif(cx<T>* b, const cx<T>* __restrict__ tws, int lt, int bar, Load ld) {
        static_assert(sizeof(T) == 4, "split-precision stages are FP32 only");
        dif_first<N, R1, TL, INV, T>(b, tws, lt, ld);
        group_sync<TL>(bar);
        dif_run<N, N / R1, TL, INV, T, OFF, kSplitSwz<N>, 8, 8>(b, tws, lt, bar);
        dft8_line<N, TL, INV, PREC>(b, lt);
        group_sync<TL>(bar);
    }
    template <bool INV, typename T, class Store>
    static __device__ __forceinline__ void dit(cx<T>* b, const cx<T>* __restrict__ tws, int lt, int bar, Store st) {
        static_assert(sizeof(T) == 4, "split-precision stages are FP32 only");
        dft8_line<N, TL, INV, PREC>(b, lt);
        group_sync<TL>(bar);
        dit_run<N, N / R1, TL, INV, T, OFF, kSplitSwz<N>, 8, 8>(b, tws, lt, bar);
        dit_last<N, R1, TL, INV, T>(b, tws, lt, st);
    }
    template <bool INV, typename T, class Store>
    static __device__ __forceinline__ void dit_blk(cx<T>* b, const cx<T>* __restrict__ tws, int tid, int nt,
                                                   Store st) {
        static_assert(sizeof(T) == 4, "split-precision stages are FP32 only");
        dft8_line_blk<N, INV, PREC>(b, tid, nt);
        __syncthreads();
        dit_run_blk<N, N / R1, INV, T, OFF, kSplitSwz<N>, 8, 8>(b, tws, tid, nt);
        dit_last_blk<N, R1, INV, T>(b, tws, tid, nt, st);
    }
    template <int TLB, bool INV, typename T, class Store>
    static __device__ __forceinline__ void dit_wide(cx<T>* b, const cx<T>* __restrict__ tws, int tid, int bar,
                                                    Store st) {
        static_assert(sizeof(T) == 4, "split-precision stages are FP32 only");
        dft8_line_blk<N, INV, PREC>(b, tid, TLB);
        wide_sync<TLB>(bar);
        dit_run_w<N, N / R1, TLB, INV, T, OFF, kSplitSwz<N>, 8, 8>(b, tws, tid, bar);
        dit_last_w<N, R1, TLB, INV, T>(b, tws, tid, st);
    }
};
template <> struct IPlan<1536, SPLIT_BF16> : IPlanSplit<1536, SPLIT_BF16> {};
template <> struct IPlan<3072, SPLIT_BF16> : IPlanSplit<3072, SPLIT_BF16> {};
template <> struct IPlan<1536, SPLIT_FP16> : IPlanSplit<1536, SPLIT_FP16> {};
template <> struct IPlan<3072, SPLIT_FP16> : IPlanSplit<3072, SPLIT_FP16> {};

}  // namespace zk
