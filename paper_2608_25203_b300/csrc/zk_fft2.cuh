// zk_fft2.cuh - in-place digit-reversing line FFTs for the right-hand-side kernels.
//
// Decimation in frequency (DIF) takes a line in natural order and leaves its
// transform in mixed-radix digit-reversed order; decimation in time (DIT)
// takes digit-reversed input and produces natural order. Every stage works in
// place: a butterfly reads R elements and writes its R results to the same
// slots, so a thread holds only R complex values and stages need one group
// barrier each.
//
// The right-hand side uses this pairing so that no reordering pass exists:
// spectra are always in natural order (where the Fourier multipliers of
// Sec. 3.2 and the truncation of Sec. 6.1 are applied), and physical values
// on the 3/2 grid are always in digit-reversed order. Pointwise products do
// not depend on the order, and every kernel that touches physical positions
// (the row kernels, the column-space fields, the series accumulator) uses the
// same plan, so the permutation cancels between an inverse (DIF) and the
// following forward (DIT) transform.
//
// Stage with block size B and radix R (SUB = B/R): butterfly b has block
// b/SUB and offset n1 = b mod SUB; it touches elements blk*B + n1 + m*SUB.
// DIF: DFT_R then multiply output m by w_B^{n1 m}; DIT: multiply input m by
// w_B^{n1 m} then DFT_R; DIT runs the stages in reverse order.
#pragma once

#include "zk_fft.cuh"

namespace zk {

// Shared-memory slot of element blk*B + n1 + m*SUB (n1 < SUB) of a stage. The
// pad-per-16 layout lets each butterfly compute one base slot and add
// compile-time offsets in three cases: SUB a multiple of 16; SUB dividing 16
// inside 16-aligned blocks; blocks of 16/B elements (last stages).
template <int B, int SUB>
__device__ __forceinline__ int stage_pbase(int blk, int n1) {
    if constexpr (SUB % 16 == 0) return pidx(blk * B + n1);
    else if constexpr (SUB < 16 && 16 % SUB == 0 && B % 16 == 0) return blk * (B + B / 16) + n1;
    else if constexpr (B < 16 && 16 % B == 0 && SUB == 1) return blk * B + ((blk * B) >> 4);
    else return 0;
}
template <int B, int SUB>
__device__ __forceinline__ int stage_slot(int pb, int base, int m) {
    if constexpr (SUB % 16 == 0) return pb + m * (SUB + SUB / 16);
    else if constexpr (SUB < 16 && 16 % SUB == 0 && B % 16 == 0) return pb + m * SUB + ((m * SUB) >> 4);
    else if constexpr (B < 16 && 16 % B == 0 && SUB == 1) return pb + m;
    else return pidx(base + m * SUB);
}

// Thread order of the radix-8 stages whose sub-blocks are narrower than 16 (SUB = 2, 4, 8):
// in the natural order the 16/SUB blocks a half-warp touches start at block offsets
// blk * B/16 (mod 16 slots) that overlap, a 2-way bank conflict on every 64-bit access.
// Moving lane bit 4 below the block bits hands each half-warp every other block, whose
// offsets are SUB slots apart, so its 16 accesses cover all 32 banks. The permutation
// stays inside each warp and keeps n1 = lane mod SUB (the fixed twiddles). The stage
// runners' SWZ switch keeps the natural order instead (the split-precision plans below 3072
// points: with the swizzle ptxas gave their 1536-point row kernels 100 registers, not 64).
template <int B, int R, int SUB>
__host__ __device__ constexpr bool stage_swizzled() {
    return R == 8 && SUB >= 2 && SUB < 16 && 16 % SUB == 0 && B % 16 == 0;
}
template <int SUB>
__device__ __forceinline__ int swz_lane(int t) {
    constexpr int LS = SUB == 2 ? 1 : SUB == 4 ? 2 : 3;   // log2 SUB
    constexpr int LH = 4 - LS;                            // log2 of the blocks per half-warp
    const int lo = t & 31, j = lo >> LS;
    const int jn = ((j & ((1 << LH) - 1)) << 1) | (j >> LH);
    return (t & ~31) | (jn << LS) | (lo & (SUB - 1));
}

// Twiddles: one table per plan holding, stage after stage, w_B^{n1 m} at
// [(m-1) * SUB + n1] (m = 1..R-1, n1 < SUB), so a warp's loads for one m are
// contiguous. OFF is the stage's offset in that table.
template <int N, int B, int R, int TL, bool INV, typename T, int OFF, bool SWZ = true>
__device__ __forceinline__ void dif_stage(cx<T>* buf, const cx<T>* __restrict__ tws, int lt) {
    constexpr int SUB = B / R, NB = N / R;
    static_assert(NB % TL == 0, "line group width must divide N/R");
    // when TL is a multiple of SUB every butterfly of this thread has the same
    // n1 = lt mod SUB: its R-1 twiddles are loaded once, before the loop
    constexpr bool FIXED = (SUB > 1) && (TL % SUB == 0);
    cx<T> wf[R > 1 ? R - 1 : 1];
    if constexpr (FIXED) {
#pragma unroll
        for (int m = 1; m < R; ++m) wf[m - 1] = __ldg(&tws[OFF + (m - 1) * SUB + lt % SUB]);
    }
    const int lts = (SWZ && stage_swizzled<B, R, SUB>() && TL % 32 == 0) ? swz_lane<SUB>(lt) : lt;
#pragma unroll
    for (int p = 0; p < NB / TL; ++p) {
        const int b = lts + p * TL;
        const int blk = b / SUB, n1 = b - blk * SUB;
        const int base = blk * B + n1;
        const int pb = stage_pbase<B, SUB>(blk, n1);
        cx<T> v[R];
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = buf[stage_slot<B, SUB>(pb, base, m)];
        SmallDFT<R, INV, T>::run(v);
        if (SUB > 1) {
#pragma unroll
            for (int m = 1; m < R; ++m)
                v[m] = cmulc<INV>(v[m], FIXED ? wf[m - 1] : __ldg(&tws[OFF + (m - 1) * SUB + n1]));
        }
#pragma unroll
        for (int m = 0; m < R; ++m) buf[stage_slot<B, SUB>(pb, base, m)] = v[m];
    }
}

template <int N, int B, int R, int TL, bool INV, typename T, int OFF, bool SWZ = true>
__device__ __forceinline__ void dit_stage(cx<T>* buf, const cx<T>* __restrict__ tws, int lt) {
    constexpr int SUB = B / R, NB = N / R;
    static_assert(NB % TL == 0, "line group width must divide N/R");
    // when TL is a multiple of SUB every butterfly of this thread has the same
    // n1 = lt mod SUB: its R-1 twiddles are loaded once, before the loop
    constexpr bool FIXED = (SUB > 1) && (TL % SUB == 0);
    cx<T> wf[R > 1 ? R - 1 : 1];
    if constexpr (FIXED) {
#pragma unroll
        for (int m = 1; m < R; ++m) wf[m - 1] = __ldg(&tws[OFF + (m - 1) * SUB + lt % SUB]);
    }
    const int lts = (SWZ && stage_swizzled<B, R, SUB>() && TL % 32 == 0) ? swz_lane<SUB>(lt) : lt;
#pragma unroll
    for (int p = 0; p < NB / TL; ++p) {
        const int b = lts + p * TL;
        const int blk = b / SUB, n1 = b - blk * SUB;
        const int base = blk * B + n1;
        const int pb = stage_pbase<B, SUB>(blk, n1);
        cx<T> v[R];
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = buf[stage_slot<B, SUB>(pb, base, m)];
        if (SUB > 1) {
#pragma unroll
            for (int m = 1; m < R; ++m)
                v[m] = cmulc<INV>(v[m], FIXED ? wf[m - 1] : __ldg(&tws[OFF + (m - 1) * SUB + n1]));
        }
        SmallDFT<R, INV, T>::run(v);
#pragma unroll
        for (int m = 0; m < R; ++m) buf[stage_slot<B, SUB>(pb, base, m)] = v[m];
    }
}

// First DIF stage (block N, table offset 0) reading its inputs through ld(p).
template <int N, int R, int TL, bool INV, typename T, class Load>
__device__ __forceinline__ void dif_first(cx<T>* buf, const cx<T>* __restrict__ tws, int lt, Load ld) {
    constexpr int SUB = N / R;
    static_assert(SUB % TL == 0, "line group width must divide N/R");
#pragma unroll 2
    for (int p = 0; p < SUB / TL; ++p) {
        const int n1 = lt + p * TL;
        cx<T> v[R];
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = ld(n1 + m * SUB, m * SUB);
        SmallDFT<R, INV, T>::run(v);
#pragma unroll
        for (int m = 1; m < R; ++m) v[m] = cmulc<INV>(v[m], __ldg(&tws[(m - 1) * SUB + n1]));
        const int pb = stage_pbase<N, SUB>(0, n1);
#pragma unroll
        for (int m = 0; m < R; ++m) buf[stage_slot<N, SUB>(pb, n1, m)] = v[m];
    }
}

// Last DIT stage (block N): hands natural-order results to st(k, value).
template <int N, int R, int TL, bool INV, typename T, class Store>
__device__ __forceinline__ void dit_last(const cx<T>* buf, const cx<T>* __restrict__ tws, int lt, Store st) {
    constexpr int SUB = N / R;
    static_assert(SUB % TL == 0, "line group width must divide N/R");
#pragma unroll 2
    for (int p = 0; p < SUB / TL; ++p) {
        const int n1 = lt + p * TL;
        cx<T> v[R];
        const int pb = stage_pbase<N, SUB>(0, n1);
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = buf[stage_slot<N, SUB>(pb, n1, m)];
#pragma unroll
        for (int m = 1; m < R; ++m) v[m] = cmulc<INV>(v[m], __ldg(&tws[(m - 1) * SUB + n1]));
        SmallDFT<R, INV, T>::run(v);
#pragma unroll
        for (int m = 0; m < R; ++m) st(n1 + m * SUB, v[m]);
    }
}

template <int N, int B, int TL, bool INV, typename T, int OFF, bool SWZ, int R, int... Rest>
__device__ __forceinline__ void dif_run(cx<T>* buf, const cx<T>* __restrict__ tws, int lt, int bar) {
    dif_stage<N, B, R, TL, INV, T, OFF, SWZ>(buf, tws, lt);
    group_sync<TL>(bar);
    if constexpr (sizeof...(Rest) > 0)
        dif_run<N, B / R, TL, INV, T, OFF + (R - 1) * (B / R), SWZ, Rest...>(buf, tws, lt, bar);
}

template <int N, int B, int TL, bool INV, typename T, int OFF, bool SWZ, int R, int... Rest>
__device__ __forceinline__ void dit_run(cx<T>* buf, const cx<T>* __restrict__ tws, int lt, int bar) {
    if constexpr (sizeof...(Rest) > 0)
        dit_run<N, B / R, TL, INV, T, OFF + (R - 1) * (B / R), SWZ, Rest...>(buf, tws, lt, bar);
    dit_stage<N, B, R, TL, INV, T, OFF, SWZ>(buf, tws, lt);
    group_sync<TL>(bar);
}

// ---- whole-block variants: every thread of the block works on one line ----
// (nt = blockDim.x threads, __syncthreads between stages). Used where one
// line must be transformed while the rest of the block would otherwise idle.
template <int N, int B, int R, bool INV, typename T, int OFF, bool SWZ = true>
__device__ __forceinline__ void dit_stage_blk(cx<T>* buf, const cx<T>* __restrict__ tws, int tid, int nt) {
    constexpr int SUB = B / R, NB = N / R;
    const int tds = (SWZ && stage_swizzled<B, R, SUB>() && NB % 32 == 0 && nt % 32 == 0) ? swz_lane<SUB>(tid) : tid;
    for (int b = tds; b < NB; b += nt) {
        const int blk = b / SUB, n1 = b - blk * SUB;
        const int base = blk * B + n1;
        const int pb = stage_pbase<B, SUB>(blk, n1);
        cx<T> v[R];
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = buf[stage_slot<B, SUB>(pb, base, m)];
        if (SUB > 1) {
#pragma unroll
            for (int m = 1; m < R; ++m) v[m] = cmulc<INV>(v[m], __ldg(&tws[OFF + (m - 1) * SUB + n1]));
        }
        SmallDFT<R, INV, T>::run(v);
#pragma unroll
        for (int m = 0; m < R; ++m) buf[stage_slot<B, SUB>(pb, base, m)] = v[m];
    }
}

template <int N, int B, bool INV, typename T, int OFF, bool SWZ, int R, int... Rest>
__device__ __forceinline__ void dit_run_blk(cx<T>* buf, const cx<T>* __restrict__ tws, int tid, int nt) {
    if constexpr (sizeof...(Rest) > 0)
        dit_run_blk<N, B / R, INV, T, OFF + (R - 1) * (B / R), SWZ, Rest...>(buf, tws, tid, nt);
    dit_stage_blk<N, B, R, INV, T, OFF, SWZ>(buf, tws, tid, nt);
    __syncthreads();
}

template <int N, int R, bool INV, typename T, class Store>
__device__ __forceinline__ void dit_last_blk(const cx<T>* buf, const cx<T>* __restrict__ tws, int tid, int nt,
                                             Store st) {
    constexpr int SUB = N / R;
    for (int n1 = tid; n1 < SUB; n1 += nt) {
        cx<T> v[R];
        const int pb = stage_pbase<N, SUB>(0, n1);
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = buf[stage_slot<N, SUB>(pb, n1, m)];
#pragma unroll
        for (int m = 1; m < R; ++m) v[m] = cmulc<INV>(v[m], __ldg(&tws[(m - 1) * SUB + n1]));
        SmallDFT<R, INV, T>::run(v);
#pragma unroll
        for (int m = 0; m < R; ++m) st(n1 + m * SUB, v[m]);
    }
}

// ---- wide-group variants: a group of TLB threads (whole warps, compile-time
// width, named barrier `bar`) transforms one line; TLB need not divide N/R
// (threads past N/R idle in that stage). Used by the row kernel's forward
// transform, where one line is shared by the threads of several line groups.
template <int TLB>
__device__ __forceinline__ void wide_sync(int bar) {
    if (bar < 0) __syncthreads();   // the group is the whole block (see group_sync)
    else asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(TLB) : "memory");
}

// SWZ: the swizzled order of the 8-wide radix-8 stage, taken only where the line does not
// divide evenly among the group's threads. Elsewhere in the wide stages, and in the 1536-point
// split-precision plans, it raised ptxas's register count of the whole row kernel (1536-point
// rows: 64 -> 100 registers, a third fewer blocks per SM), which cost more than the bank
// conflict.
template <int N, int B, int R, int TLB, bool INV, typename T, int OFF, bool SWZ = true>
__device__ __forceinline__ void dit_stage_w(cx<T>* buf, const cx<T>* __restrict__ tws, int tid) {
    constexpr int SUB = B / R, NB = N / R;
    constexpr int PER = (NB + TLB - 1) / TLB;
    constexpr bool EVEN = NB % TLB == 0;
    constexpr bool FIXED = (SUB > 1) && EVEN && (TLB % SUB == 0);
    cx<T> wf[R > 1 ? R - 1 : 1];
    if constexpr (FIXED) {
#pragma unroll
        for (int m = 1; m < R; ++m) wf[m - 1] = __ldg(&tws[OFF + (m - 1) * SUB + tid % SUB]);
    }
    const int tds = (SWZ && stage_swizzled<B, R, SUB>() && !EVEN && TLB % 32 == 0 && NB % 32 == 0) ? swz_lane<SUB>(tid) : tid;
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int b = tds + p * TLB;
        if (EVEN || b < NB) {
            const int blk = b / SUB, n1 = b - blk * SUB;
            const int base = blk * B + n1;
            const int pb = stage_pbase<B, SUB>(blk, n1);
            cx<T> v[R];
#pragma unroll
            for (int m = 0; m < R; ++m) v[m] = buf[stage_slot<B, SUB>(pb, base, m)];
            if constexpr (SUB > 1) {
#pragma unroll
                for (int m = 1; m < R; ++m)
                    v[m] = cmulc<INV>(v[m], FIXED ? wf[m - 1] : __ldg(&tws[OFF + (m - 1) * SUB + n1]));
            }
            SmallDFT<R, INV, T>::run(v);
#pragma unroll
            for (int m = 0; m < R; ++m) buf[stage_slot<B, SUB>(pb, base, m)] = v[m];
        }
    }
}

template <int N, int B, int TLB, bool INV, typename T, int OFF, bool SWZ, int R, int... Rest>
__device__ __forceinline__ void dit_run_w(cx<T>* buf, const cx<T>* __restrict__ tws, int tid, int bar) {
    if constexpr (sizeof...(Rest) > 0)
        dit_run_w<N, B / R, TLB, INV, T, OFF + (R - 1) * (B / R), SWZ, Rest...>(buf, tws, tid, bar);
    dit_stage_w<N, B, R, TLB, INV, T, OFF, SWZ>(buf, tws, tid);
    wide_sync<TLB>(bar);
}

template <int N, int R, int TLB, bool INV, typename T, class Store>
__device__ __forceinline__ void dit_last_w(const cx<T>* buf, const cx<T>* __restrict__ tws, int tid, Store st) {
    constexpr int SUB = N / R;
    constexpr int PER = (SUB + TLB - 1) / TLB;
    constexpr bool EVEN = SUB % TLB == 0;
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int n1 = tid + p * TLB;
        if (EVEN || n1 < SUB) {
            cx<T> v[R];
            const int pb = stage_pbase<N, SUB>(0, n1);
#pragma unroll
            for (int m = 0; m < R; ++m) v[m] = buf[stage_slot<N, SUB>(pb, n1, m)];
#pragma unroll
            for (int m = 1; m < R; ++m) v[m] = cmulc<INV>(v[m], __ldg(&tws[(m - 1) * SUB + n1]));
            SmallDFT<R, INV, T>::run(v);
#pragma unroll
            for (int m = 0; m < R; ++m) st(n1 + m * SUB, v[m]);
        }
    }
}

// Plans for the 3/2-padded line lengths: line-group width TL and radices in
// DIF order. The last DIF stage is radix 16 (or 8 for the smallest line):
// its stride-16 groups land on distinct banks with the pad-per-16 layout,
// and TL divides N/R for every radix.
//
// Variant V = 0 is the default plan of each length. V = 1 is an alternative
// for the long lines (radix 16 throughout, half the line-group width of the
// radix-8 plan at the same shared memory per line); for the short lines it is
// the default plan again. The batch autotuner times both per tile shape.
template <int N, int V = 0> struct IPlan;
#define ZK_IPLAN(N_, V_, TL_, R1_, ...)                                                                  \
    template <> struct IPlan<N_, V_> {                                                                   \
        static constexpr int TL = TL_, R1 = R1_;                                                         \
        static constexpr int RADICES[] = {R1_, __VA_ARGS__};                                             \
        static constexpr int NSTAGE = sizeof(RADICES) / sizeof(int);                                     \
        template <bool INV, typename T, class Load>                                                      \
        static __device__ __forceinline__ void dif(cx<T>* b, const cx<T>* __restrict__ tws, int lt,      \
                                                   int bar, Load ld) {                                   \
            dif_first<N_, R1_, TL_, INV, T>(b, tws, lt, ld);                                             \
            group_sync<TL_>(bar);                                                                        \
            dif_run<N_, N_ / R1_, TL_, INV, T, (R1_ - 1) * (N_ / R1_), true, __VA_ARGS__>(b, tws, lt, bar); \
        }                                                                                                \
        template <bool INV, typename T, class Store>                                                     \
        static __device__ __forceinline__ void dit(cx<T>* b, const cx<T>* __restrict__ tws, int lt,      \
                                                   int bar, Store st) {                                  \
            dit_run<N_, N_ / R1_, TL_, INV, T, (R1_ - 1) * (N_ / R1_), true, __VA_ARGS__>(b, tws, lt, bar); \
            dit_last<N_, R1_, TL_, INV, T>(b, tws, lt, st);                                              \
        }                                                                                                \
        template <bool INV, typename T, class Store>                                                     \
        static __device__ __forceinline__ void dit_blk(cx<T>* b, const cx<T>* __restrict__ tws, int tid, \
                                                       int nt, Store st) {                               \
            dit_run_blk<N_, N_ / R1_, INV, T, (R1_ - 1) * (N_ / R1_), true, __VA_ARGS__>(b, tws, tid, nt); \
            dit_last_blk<N_, R1_, INV, T>(b, tws, tid, nt, st);                                          \
        }                                                                                                \
        template <int TLB, bool INV, typename T, class Store>                                            \
        static __device__ __forceinline__ void dit_wide(cx<T>* b, const cx<T>* __restrict__ tws, int tid,\
                                                        int bar, Store st) {                             \
            dit_run_w<N_, N_ / R1_, TLB, INV, T, (R1_ - 1) * (N_ / R1_), true, __VA_ARGS__>(b, tws, tid, bar); \
            dit_last_w<N_, R1_, TLB, INV, T>(b, tws, tid, st);                                           \
        }                                                                                                \
    };
ZK_IPLAN(24, 0, 1, 3, 8)
ZK_IPLAN(48, 0, 1, 3, 16)
ZK_IPLAN(96, 0, 2, 6, 16)
ZK_IPLAN(192, 0, 4, 12, 16)
ZK_IPLAN(384, 0, 8, 6, 4, 16)
// radix-8 plans: every stage has N/R divisible by 128 (3072), 64 (1536) or
// 32 (768); the third stage (SUB = 8) runs in the swizzled thread order above
ZK_IPLAN(768, 0, 32, 3, 4, 8, 8)
ZK_IPLAN(1536, 0, 64, 3, 8, 8, 8)
ZK_IPLAN(3072, 0, 128, 6, 8, 8, 8)
ZK_IPLAN(768, 1, 16, 3, 16, 16)
ZK_IPLAN(1536, 1, 32, 6, 16, 16)
ZK_IPLAN(3072, 1, 64, 12, 16, 16)
#undef ZK_IPLAN
template <int N> struct IPlan<N, 1> : IPlan<N, 0> {};
// lengths whose V = 1 plan differs from the default
__host__ __device__ constexpr bool plan_has_variant(int n) { return n == 768 || n == 1536 || n == 3072; }

// Host/device description of a plan for building its twiddle table.
struct PlanDesc {
    int n, nstage, radix[4];
};
template <int N, int V = 0> __host__ __device__ constexpr PlanDesc plan_desc() {
    PlanDesc d{N, IPlan<N, V>::NSTAGE, {1, 1, 1, 1}};
    for (int i = 0; i < IPlan<N, V>::NSTAGE; ++i) d.radix[i] = IPlan<N, V>::RADICES[i];
    return d;
}
inline PlanDesc plan_desc_of(int n, int v = 0) {
    if (v == 1 && plan_has_variant(n)) {
        switch (n) {
        case 768: return plan_desc<768, 1>();
        case 1536: return plan_desc<1536, 1>();
        case 3072: return plan_desc<3072, 1>();
        default: break;
        }
    }
    switch (n) {
    case 24: return plan_desc<24>();
    case 48: return plan_desc<48>();
    case 96: return plan_desc<96>();
    case 192: return plan_desc<192>();
    case 384: return plan_desc<384>();
    case 768: return plan_desc<768>();
    case 1536: return plan_desc<1536>();
    case 3072: return plan_desc<3072>();
    default: return PlanDesc{0, 0, {1, 1, 1, 1}};
    }
}
// Half-length plan of a real line: when the plan of N starts with an even radix R1 and the plan
// of N/2 is (R1/2, same later radices), the DIF output slot s = m1 (N/R1) + r (first digit m1)
// holds the same physical position as slot (m1/2) (N/R1) + r of the N/2 plan, times two, plus
// (m1 mod 2). A real line x of N points can then be packed as z[n] = x[2n] + i x[2n+1] with no
// reordering and transformed at half length (the forward real-input transform of the row
// rounds). Host and device read the same plan descriptions.
inline __host__ __device__ constexpr bool half_plan_match(const PlanDesc& d, const PlanDesc& h) {
    if (d.n < 48 || d.n % 2 != 0 || h.n * 2 != d.n || d.nstage != h.nstage) return false;
    if (d.radix[0] % 2 != 0 || h.radix[0] * 2 != d.radix[0]) return false;
    for (int i = 1; i < d.nstage; ++i)
        if (d.radix[i] != h.radix[i]) return false;
    return true;
}
template <int N, int V> __host__ __device__ constexpr bool half_plan_ok() {
    if constexpr (N < 48 || N % 2 != 0 || (V != 0 && V != 1)) return false;
    else return half_plan_match(plan_desc<N, V>(), plan_desc<N / 2, V>());
}
inline bool half_plan_ok_host(int n, int v) {
    if (n < 48 || n % 2 != 0 || (v != 0 && v != 1)) return false;
    const PlanDesc d = plan_desc_of(n, v), h = plan_desc_of(n / 2, v);
    return d.n == n && h.n == n / 2 && half_plan_match(d, h);
}

// Number of table entries, and entry e as (numerator, B) of the angle -2 pi num / B.
inline int plan_table_size(const PlanDesc& d) {
    int n = 0, B = d.n;
    for (int s = 0; s < d.nstage; ++s) { n += (d.radix[s] - 1) * (B / d.radix[s]); B /= d.radix[s]; }
    return n;
}
__host__ __device__ inline void plan_table_entry(const PlanDesc& d, int e, long long* num, int* den) {
    int B = d.n;
    for (int s = 0; s < d.nstage; ++s) {
        const int R = d.radix[s], SUB = B / R, cnt = (R - 1) * SUB;
        if (e < cnt) {
            const int m = 1 + e / SUB, n1 = e % SUB;
            *num = ((long long)n1 * m) % B;
            *den = B;
            return;
        }
        e -= cnt;
        B /= R;
    }
    *num = 0;
    *den = 1;
}

}  // namespace zk
