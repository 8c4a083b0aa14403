// zk_fft.cuh - shared-memory line FFTs for the Zakharov step (sm_103a).
//
// Every spectral operator of the method (Sec. 3.2: G0, B0, grad and the dz^a
// symbols; Sec. 6.1: 3/2 zero padding and truncation) is applied between
// discrete Fourier transforms of grid lines. This file holds the transform
// engine: a mixed-radix Stockham FFT of one line held in shared memory,
// computed cooperatively by a "line group" of TL threads.
//
//  * Convention: forward X[k] = sum_j x[j] exp(-2 pi i j k / N); the inverse
//    flips the sign and applies no 1/N factor (callers fold all scale
//    factors into their spectral multipliers).
//  * Stockham stage with radix R after sub-transforms of length L are done:
//    butterfly b (0 <= b < N/R), j = b mod L, k = b / L reads x[b + m N/R],
//    m < R, twiddles input m by w_{LR}^{j m}, runs a length-R DFT in
//    registers and writes x[k L R + j + m L]. Stages run in place: every
//    thread of the group reads all its inputs, the group synchronises, then
//    writes. The result comes out in natural order.
//  * Shared-memory layout of a line: element i lives at i + i/16 (one pad
//    slot per 16 complex values) so the strided stage writes of the first
//    stage spread over all banks.
//  * Twiddles w_N^t, t < N, come from a table in global memory built on the
//    host in FP64 (read through the read-only cache); the constants inside
//    the small DFTs are cos/sin of multiples of 2 pi / 48, written out below.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace zk {

template <typename T> struct CT;
template <> struct CT<float> { using type = float2; };
template <> struct CT<double> { using type = double2; };
template <typename T> using cx = typename CT<T>::type;

template <typename T> __host__ __device__ __forceinline__ cx<T> mk(T a, T b) { cx<T> r; r.x = a; r.y = b; return r; }
template <typename V> __host__ __device__ __forceinline__ V cadd(V a, V b) { a.x += b.x; a.y += b.y; return a; }
template <typename V> __host__ __device__ __forceinline__ V csub(V a, V b) { a.x -= b.x; a.y -= b.y; return a; }
// FP32 complex add and subtract as one packed instruction each (add/sub.rn.f32x2: two IEEE
// round-to-nearest operations, the same results as the scalar pair); the butterflies issue
// fewer instructions, which is what bounds the transforms.
#ifdef __CUDA_ARCH__
__device__ __forceinline__ unsigned long long f2_pack(float2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 f2_unpack(unsigned long long r) {
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
#endif
template <> __host__ __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
    return f2_unpack(r);
#else
    a.x += b.x; a.y += b.y; return a;
#endif
}
template <> __host__ __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
    return f2_unpack(r);
#else
    a.x -= b.x; a.y -= b.y; return a;
#endif
}
template <typename V, typename S> __host__ __device__ __forceinline__ V cscale(V a, S s) { a.x *= s; a.y *= s; return a; }
template <typename V> __host__ __device__ __forceinline__ V cmul(V a, V b) {
    V r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename V> __host__ __device__ __forceinline__ V cconj(V a) { a.y = -a.y; return a; }
// multiply by +i
template <typename V> __host__ __device__ __forceinline__ V cmuli(V a) { V r; r.x = -a.y; r.y = a.x; return r; }
// multiply by -i
template <typename V> __host__ __device__ __forceinline__ V cmulmi(V a) { V r; r.x = a.y; r.y = -a.x; return r; }
// multiply by a conj(b) if INV else by b
template <bool CONJ, typename V> __host__ __device__ __forceinline__ V cmulc(V a, V b) {
    V r;
    if (CONJ) { r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; }
    else      { r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; }
    return r;
}

// cos(2 pi j / 48), j = 0..12 (first quadrant); the rest follows by symmetry.
__host__ __device__ constexpr double c48q(int r) {
    return r == 0 ? 1.0 : r == 1 ? 0.9914448613738104111445575 : r == 2 ? 0.9659258262890682867497432
         : r == 3 ? 0.9238795325112867561281832 : r == 4 ? 0.8660254037844386467637232
         : r == 5 ? 0.793353340291235164579777  : r == 6 ? 0.7071067811865475244008444
         : r == 7 ? 0.6087614290087206394160975 : r == 8 ? 0.5
         : r == 9 ? 0.38268343236508977172846   : r == 10 ? 0.2588190451025207623488988
         : r == 11 ? 0.1305261922200515915484062 : 0.0;
}
__host__ __device__ constexpr double c48(int j) {
    // j taken mod 48
    return ((j % 48 + 48) % 48) / 12 == 0 ? c48q((j % 48 + 48) % 48)
         : ((j % 48 + 48) % 48) / 12 == 1 ? -c48q(12 - (j % 48 + 48) % 48 % 12)
         : ((j % 48 + 48) % 48) / 12 == 2 ? -c48q((j % 48 + 48) % 48 % 12)
         : c48q(12 - (j % 48 + 48) % 48 % 12);
}
__host__ __device__ constexpr double s48(int j) { return c48(j - 12); }

// a * exp(-+ 2 pi i e / R) with e a compile-time constant after unrolling.
template <int R, bool INV, typename T>
__device__ __forceinline__ cx<T> twc(cx<T> a, int e) {
    const int q = ((e % R) + R) % R;
    if (q == 0) return a;
    const int j = q * (48 / R);              // angle 2 pi j / 48
    if (j == 12) return INV ? cmuli(a) : cmulmi(a);
    if (j == 24) return mk<T>(-a.x, -a.y);
    if (j == 36) return INV ? cmulmi(a) : cmuli(a);
    const T c = (T)c48(j);
    const T s = INV ? (T)s48(j) : (T)(-s48(j));
    return mk<T>(a.x * c - a.y * s, a.x * s + a.y * c);
}

// ---- small DFTs in registers (natural order in and out) --------------------
template <int R, bool INV, typename T> struct SmallDFT;

template <bool INV, typename T> struct SmallDFT<1, INV, T> {
    static __device__ __forceinline__ void run(cx<T>*) {}
};
template <bool INV, typename T> struct SmallDFT<2, INV, T> {
    static __device__ __forceinline__ void run(cx<T>* v) {
        cx<T> a = v[0];
        v[0] = cadd(a, v[1]); v[1] = csub(a, v[1]);
    }
};
template <bool INV, typename T> struct SmallDFT<3, INV, T> {
    static __device__ __forceinline__ void run(cx<T>* v) {
        const T s = INV ? (T)0.866025403784438646763723170752936183 : (T)-0.866025403784438646763723170752936183;
        cx<T> t1 = cadd(v[1], v[2]);
        cx<T> t2 = csub(v[0], cscale(t1, (T)0.5));
        cx<T> d = csub(v[1], v[2]);
        cx<T> t3 = mk<T>(-s * d.y, s * d.x);
        v[0] = cadd(v[0], t1); v[1] = cadd(t2, t3); v[2] = csub(t2, t3);
    }
};
template <bool INV, typename T> struct SmallDFT<4, INV, T> {
    static __device__ __forceinline__ void run(cx<T>* v) {
        cx<T> a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
        cx<T> a2 = cadd(v[1], v[3]);
        cx<T> d = csub(v[1], v[3]);
        cx<T> a3 = INV ? cmuli(d) : cmulmi(d);
        v[0] = cadd(a0, a2); v[2] = csub(a0, a2); v[1] = cadd(a1, a3); v[3] = csub(a1, a3);
    }
};
// Cooley-Tukey split R = R1 * R2 with constant inner twiddles.
template <int R1, int R2, bool INV, typename T>
__device__ __forceinline__ void dft_ct(cx<T>* v) {
    constexpr int R = R1 * R2;
    cx<T> y[R];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) {
        cx<T> t[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) t[n1] = v[R2 * n1 + n2];
        SmallDFT<R1, INV, T>::run(t);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) y[n2 * R1 + k1] = twc<R, INV, T>(t[k1], n2 * k1);
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
        cx<T> t[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) t[n2] = y[n2 * R1 + k1];
        SmallDFT<R2, INV, T>::run(t);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = t[k2];
    }
}
template <bool INV, typename T> struct SmallDFT<6, INV, T> {
    static __device__ __forceinline__ void run(cx<T>* v) { dft_ct<2, 3, INV, T>(v); }
};
template <bool INV, typename T> struct SmallDFT<8, INV, T> {
    static __device__ __forceinline__ void run(cx<T>* v) { dft_ct<2, 4, INV, T>(v); }
};
template <bool INV, typename T> struct SmallDFT<12, INV, T> {
    static __device__ __forceinline__ void run(cx<T>* v) { dft_ct<4, 3, INV, T>(v); }
};
template <bool INV, typename T> struct SmallDFT<16, INV, T> {
    static __device__ __forceinline__ void run(cx<T>* v) { dft_ct<4, 4, INV, T>(v); }
};

// ---- line layout and group synchronisation --------------------------------
__host__ __device__ constexpr int pidx(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int line_stride(int N) { return N + (N >> 4) + 1; }

// A negative barrier id stands for the whole block (a block of exactly one line group). Kernels
// that pass a constant -1 then use barrier 0 alone: the named barriers a block reserves (16 when
// the id is a run-time value) cap how many blocks an SM holds.
template <int TL>
__device__ __forceinline__ void group_sync(int bar) {
    if constexpr (TL > 32) {
        if (bar < 0) __syncthreads();
        else asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(TL) : "memory");
    } else {
        __syncwarp();
    }
}

// One Stockham stage of radix R on a line of N after length-L sub-transforms.
template <int N, int R, int L, int TL, bool INV, typename T>
__device__ __forceinline__ void fft_stage(cx<T>* buf, const cx<T>* __restrict__ tw, int lt, int bar) {
    constexpr int NB = N / R;
    constexpr int PER = (NB + TL - 1) / TL;
    constexpr int S = N / (L * R);
    cx<T> v[PER][R];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int b = lt + p * TL;
        if ((NB % TL == 0) || b < NB) {
#pragma unroll
            for (int m = 0; m < R; ++m) v[p][m] = buf[pidx(b + m * NB)];
        }
    }
    group_sync<TL>(bar);
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int b = lt + p * TL;
        if ((NB % TL == 0) || b < NB) {
            const int j = (L == 1) ? 0 : (b % L);
            const int k = (L == 1) ? b : (b / L);
            if (L > 1) {
#pragma unroll
                for (int m = 1; m < R; ++m) v[p][m] = cmulc<INV>(v[p][m], __ldg(&tw[j * m * S]));
            }
            SmallDFT<R, INV, T>::run(v[p]);
#pragma unroll
            for (int m = 0; m < R; ++m) buf[pidx(k * L * R + j + m * L)] = v[p][m];
        }
    }
    group_sync<TL>(bar);
}

template <int N, int L, bool INV, typename T, int TL, int R, int... Rest>
__device__ __forceinline__ void run_stages(cx<T>* buf, const cx<T>* __restrict__ tw, int lt, int bar) {
    fft_stage<N, R, L, TL, INV, T>(buf, tw, lt, bar);
    if constexpr (sizeof...(Rest) > 0) run_stages<N, L * R, INV, T, TL, Rest...>(buf, tw, lt, bar);
}

// Radix plan and line-group width per transform length. The width TL divides
// N/R for the large radices so that every thread does the same number of
// butterflies per stage; per-thread register use stays at <= 48 complex values.
template <int N> struct Plan;
#define ZK_PLAN(N_, TL_, ...)                                                                   \
    template <> struct Plan<N_> {                                                               \
        static constexpr int TL = TL_;                                                          \
        template <bool INV, typename T>                                                         \
        static __device__ __forceinline__ void run(cx<T>* b, const cx<T>* __restrict__ tw,      \
                                                   int lt, int bar) {                           \
            run_stages<N_, 1, INV, T, TL_, __VA_ARGS__>(b, tw, lt, bar);                        \
        }                                                                                       \
    };
ZK_PLAN(16, 1, 16)
ZK_PLAN(24, 1, 8, 3)
ZK_PLAN(32, 1, 4, 8)
ZK_PLAN(48, 1, 4, 12)
ZK_PLAN(64, 2, 8, 8)
ZK_PLAN(96, 2, 8, 12)
ZK_PLAN(128, 4, 8, 16)
ZK_PLAN(192, 4, 16, 12)
ZK_PLAN(256, 8, 16, 16)
ZK_PLAN(384, 8, 8, 4, 12)
ZK_PLAN(512, 16, 8, 8, 8)
ZK_PLAN(768, 16, 16, 16, 3)
ZK_PLAN(1024, 32, 4, 16, 16)
ZK_PLAN(1536, 32, 16, 16, 6)
ZK_PLAN(2048, 64, 8, 16, 16)
ZK_PLAN(3072, 64, 16, 16, 12)
#undef ZK_PLAN

}  // namespace zk
