// zk_kernels2.cuh - row and column kernels of the right-hand side on the in-place
// digit-reversing FFTs of zk_fft2.cuh (same argument blocks as zk_kernels.cuh).
//
// Order conventions: column-space row zp and position p of a padded row are
// digit-reversed physical indices (written by DIF inverses, read by DIT
// forwards of the same plan); spectra (compact fields, kx of a row, kz of a
// column after a DIT) are in natural order.
#pragma once

#include "zk_dftmma.cuh"
#include "zk_kernels.cuh"

namespace zk {

template <typename T> __device__ __forceinline__ T tanh_kh(T x);
// tanh(x) rounds to 1 in FP32 for x > 9.01 (1 - tanh < 2^-25) and in FP64 for x > 18.7.
template <> __device__ __forceinline__ float tanh_kh<float>(float x) { return x > 9.5f ? 1.0f : tanhf(x); }
template <> __device__ __forceinline__ double tanh_kh<double>(double x) { return x > 20.0 ? 1.0 : tanh(x); }

// |k| from |k|^2 for the DNO symbols: FP32 contexts use the hardware reciprocal square
// root (a few ulp, below the FP32 rounding of the products it scales); FP64 uses sqrt.
template <typename T> __device__ __forceinline__ T d_kabs(T k2);
template <> __device__ __forceinline__ float d_kabs<float>(float k2) { return k2 > 0.f ? k2 * rsqrtf(k2) : 0.f; }
template <> __device__ __forceinline__ double d_kabs<double>(double k2) { return sqrt(k2); }

template <typename T> __device__ __forceinline__ void d_sincos(T x, T* s, T* c);
template <> __device__ __forceinline__ void d_sincos<float>(float x, float* s, float* c) { sincosf(x, s, c); }
template <> __device__ __forceinline__ void d_sincos<double>(double x, double* s, double* c) { sincos(x, s, c); }

// Taper of Sec. 6.1, exp[-(|k|/kc)^8], from u2 = |k|^2 / kc^2. FP32 contexts use the
// hardware exponential (__expf: a few ulp near 1, far below the FP32 rounding of the
// products it multiplies); FP64 contexts use exp.
template <typename T> __device__ __forceinline__ T d_taper(T u2);
template <> __device__ __forceinline__ float d_taper<float>(float u2) {
    const float u4 = u2 * u2;
    return __expf(-(u4 * u4));
}
template <> __device__ __forceinline__ double d_taper<double>(double u2) {
    const double u4 = u2 * u2;
    return exp(-(u4 * u4));
}

// ---------------------------------------------------------------------------
// Row kernel: persistent over padded rows.
// ---------------------------------------------------------------------------
// TA: type of the series sums (the in-round W / Phi sums, the accumulator
// across orders and the final G_nl / Bernoulli assembly); T, or double for
// FP32 contexts with FP64 series accumulation (the accumulator buffer then
// holds doubles).
// Largest row-kernel block: it bounds the registers a thread may use (the
// line groups of a wider round take their lines in waves). 512 threads leave
// 128 registers: the transforms then run without register pressure, at 16
// warps per SM (measured faster than 24-32 warps at 64 registers).
#ifndef ZK_ROW_MAX_THREADS
#define ZK_ROW_MAX_THREADS 512
#endif
constexpr int kRowMaxThreads = ZK_ROW_MAX_THREADS;


// Read-once global loads: an L2 evict-first cache policy (created once per thread) keeps them
// from displacing data that is still to be used.
__device__ __forceinline__ unsigned long long l2_evict_first_policy() {
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ float ldg_evict_first(const float* p, unsigned long long pol) {
    float v;
    asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ double ldg_evict_first(const double* p, unsigned long long pol) {
    double v;
    asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}

// DIV = NPX / (nx / 2): 3 for the 3/2 rule, 6 for the 3N padding.
// ONEG: the block is a single line group (rounds with one line): every barrier is barrier 0,
// so the block reserves one hardware barrier instead of 16 and more blocks fit on an SM.
template <typename T, int NPX, int V = 0, typename TA = T, int DIV = 3, bool ONEG = false>
__global__ void __launch_bounds__(kRowMaxThreads) row2_kernel(const RowArgs<T> a, const cx<T>* __restrict__ tw) {
    using P = IPlan<NPX, V>;
    constexpr int TL = P::TL;
    constexpr int HX = NPX / DIV;
    constexpr int LS = line_stride(NPX);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* lines = reinterpret_cast<cx<T>*>(smem_raw);
    const int g = ONEG ? 0 : threadIdx.x / TL, lt = ONEG ? threadIdx.x : threadIdx.x % TL;
    const int bar = ONEG ? -1 : 1 + (g & 7);
    const int ngroups = blockDim.x / TL;
    // wide groups (TL >= 32) take lines in waves; narrow groups share warps and
    // each runs exactly one line (idle ones on zeros) so warp barriers match
    const int nloop = TL < 32 ? ngroups : a.nlines;
    const T kx0 = a.kx0;
    constexpr int SUB1 = NPX / P::R1;
    // Phi(r) (real) forward-transformed at half length: Phase B packs x[2n] + i x[2n+1] in
    // place (a position's new slot belongs to the same thread and to a position it has already
    // read, when the block width divides SUB1), Phase C runs the N/2 plan and splits the result.
    constexpr bool HALF_OK = TL >= 32 && half_plan_ok<NPX, V>();
    const bool half = HALF_OK && a.kind == 0 && a.twh != nullptr && (SUB1 % blockDim.x) == 0;
    const cx<T>* colbase = a.colbase + (long long)blockIdx.y * a.tcol;
    TA* acc = reinterpret_cast<TA*>(a.acc) + (long long)blockIdx.y * a.tacc;
    cx<T>* out0 = a.out0 + (long long)blockIdx.y * a.tcol;
    cx<T>* out1 = a.out1 ? a.out1 + (long long)blockIdx.y * a.tcol : nullptr;

    // the series accumulator row is read by rounds r >= 3 and by the final round when M >= 3
    const bool reads_acc = a.kind == 0 ? a.r >= 3 : a.M >= 3;
    // the slopes of eta enter round r when r - 1 <= M - 3, and always the final round
    const bool slopes = a.kind == 0 ? (a.r >= 2 && a.r - 1 <= a.M - 3) : true;
    const bool eta_in = a.kind == 0 || a.M >= 2;
    // surface planes of this tile: eta, dx eta, dz eta, PL elements apart
    const long long PL = (long long)a.npz * NPX;
    T* sfc = a.sfc_mode ? a.sfc + (long long)blockIdx.y * a.tsfc : nullptr;
    const int npl = a.sfc_mode == 2 ? (slopes ? 3 : (eta_in ? 1 : 0)) : 0;   // planes read
    // the planes are read once per round: their L2 lines go first, before the rows in flight
    const unsigned long long pol = l2_evict_first_policy();
    for (int zp = blockIdx.x; zp < a.npz; zp += gridDim.x) {
        // Phase A: Hermitian packing of two real fields fused into the first DIF stage.
        for (int l = g; l < nloop; l += ngroups) {
            cx<T>* lb = lines + (size_t)l * LS;
            const bool act = l < a.nlines;
            const int fa = act ? a.fa[l] : -1, fb = act ? a.fb[l] : -1;
            const bool da = act && ((a.dxa >> l) & 1u), db = act && ((a.dxb >> l) & 1u);
            const cx<T>* pa = fa >= 0 ? colbase + (long long)fa * a.fstride + (long long)zp * HX : nullptr;
            const cx<T>* pb = fb >= 0 ? colbase + (long long)fb * a.fstride + (long long)zp * HX : nullptr;
            // ms = m * SUB1 of the first stage (a compile-time constant after unrolling):
            // the zero band, and in most cases the direct / mirror choice, follow from it.
            auto ld = [&](int m, int ms) -> cx<T> {
                int mm;
                bool mir;
                if (ms + SUB1 <= HX) { mm = m; mir = false; }
                else if (ms >= HX && ms + SUB1 <= NPX - HX + 1) return mk<T>(0, 0);
                else if (ms > NPX - HX) { mm = NPX - m; mir = true; }
                else if (m < HX) { mm = m; mir = false; }
                else if (m > NPX - HX) { mm = NPX - m; mir = true; }
                else return mk<T>(0, 0);
                cx<T> A = pa ? __ldg(pa + mm) : mk<T>(0, 0);
                cx<T> B = pb ? __ldg(pb + mm) : mk<T>(0, 0);
                const T kx = kx0 * (T)mm;
                if (da) A = mk<T>(-kx * A.y, kx * A.x);
                if (db) B = mk<T>(-kx * B.y, kx * B.x);
                if (mm == 0) { A.y = 0; B.y = 0; }
                return mir ? mk<T>(A.x + B.y, B.x - A.y) : mk<T>(A.x - B.y, A.y + B.x);
            };
            P::template dif<true, T>(lb, tw, lt, bar, ld);
        }
        __syncthreads();

        // Ask L2 for this block's next row once this row's inputs are in: its input lines (HX
        // contiguous values per field), accumulator row and surface-plane rows then arrive while
        // the current row's pointwise phase and forward transform run. Issued a whole row
        // earlier, the prefetched rows of all resident blocks outgrew L2 and were partly evicted
        // before use. Sizes and addresses are multiples of 16 bytes (HX, the field stride and
        // NPX are even; NPX is a multiple of 4). Grids below 1024 points per axis keep their
        // fields in L2 and would only pay the instructions.
        const int zn = zp + gridDim.x;
        if (NPX >= 1536 && zn < a.npz && threadIdx.x <= 2 * a.nlines + npl) {
            const void* src = nullptr;
            unsigned bytes = 0;
            const int t = threadIdx.x;
            if (t < 2 * a.nlines) {
                const int l = t >> 1;
                const int f = (t & 1) ? a.fb[l] : a.fa[l];
                if (f >= 0) {
                    src = colbase + (long long)f * a.fstride + (long long)zn * HX;
                    bytes = (unsigned)(HX * sizeof(cx<T>));
                }
            } else if (t == 2 * a.nlines) {
                if (reads_acc) {
                    src = acc + (long long)zn * NPX;
                    bytes = (unsigned)(NPX * sizeof(TA));
                }
            } else {
                src = sfc + (long long)(t - 2 * a.nlines - 1) * PL + (long long)zn * NPX;
                bytes = (unsigned)(NPX * sizeof(T));
            }
            if (src) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
        }
        // Phase B: pointwise HOS terms (positions in digit-reversed order).
        auto slot = [&](int s, int p) -> T {
            const cx<T> v = lines[(s >> 1) * LS + pidx(p)];
            return (s & 1) ? v.y : v.x;
        };
        TA* accrow = acc + (long long)zp * NPX;
        T* srow = sfc ? sfc + (long long)zp * NPX : nullptr;
        // eta and its slopes at position p: from the surface planes (mode 2, preloaded into
        // se[] below) or from their slots in the transformed lines
        const bool rd_sfc = a.sfc_mode == 2;
        // PB positions per iteration: their accumulator and surface-plane reads (global
        // memory) are issued together, and the independent position updates interleave.
        constexpr int PB = 4;
        for (int p0 = threadIdx.x; p0 < NPX; p0 += PB * blockDim.x) {
            const bool rd_acc = a.kind == 0 ? a.r >= 3 : a.M >= 3;
            TA prev[PB];
            T se[3][PB];
#pragma unroll
            for (int j = 0; j < PB; ++j) {
                const int p = p0 + j * blockDim.x;
                const bool in = p < NPX;
                prev[j] = (rd_acc && in) ? accrow[p] : (TA)0;
                se[0][j] = (rd_sfc && eta_in && in) ? ldg_evict_first(srow + p, pol) : (T)0;
                se[1][j] = (rd_sfc && slopes && in) ? ldg_evict_first(srow + PL + p, pol) : (T)0;
                se[2][j] = (rd_sfc && slopes && in) ? ldg_evict_first(srow + 2 * PL + p, pol) : (T)0;
            }
            if (a.sfc_mode == 1) {
#pragma unroll
                for (int j = 0; j < PB; ++j) {
                    const int p = p0 + j * blockDim.x;
                    if (p >= NPX) break;
                    srow[p] = (T)slot(a.s_eta, p);
                    srow[PL + p] = (T)slot(a.s_etax, p);
                    srow[2 * PL + p] = (T)slot(a.s_etaz, p);
                }
            }
            if (a.kind == 0) {
                const int r = a.r;
#pragma unroll
                for (int j = 0; j < PB; ++j) {
                    const int p = p0 + j * blockDim.x;
                    if (p >= NPX) break;
                    const TA eta = rd_sfc ? (TA)se[0][j] : slot(a.s_eta, p);
                    TA W = 0, Phi = 0, ep = 1;
                    // unrolled over the largest order so that each 1/q is a constant (no division)
#pragma unroll
                    for (int q = 1; q <= kMaxOrder; ++q) {
                        if (q > r) break;
                        const TA eq = ep * eta * (TA)(1.0 / q);
                        const TA F = slot(a.s_F0 + (r - q), p);
                        W += ep * F;
                        Phi -= eq * F;
                        ep = eq;
                    }
                    if (r >= 2) {
                        TA coef = a.epsp[r - 1];
                        if (r - 1 <= a.M - 3) {
                            const TA ex = rd_sfc ? (TA)se[1][j] : slot(a.s_etax, p);
                            const TA ez = rd_sfc ? (TA)se[2][j] : slot(a.s_etaz, p);
                            coef += (TA)a.epsp[r + 1] * (ex * ex + ez * ez);
                        }
                        accrow[p] = prev[j] + coef * W;
                    }
                    if (HALF_OK && half) {
                        // slot m1 SUB1 + q of the N plan -> component (m1 mod 2) of slot
                        // (m1 / 2) SUB1 + q of the N/2 plan
                        const int m1 = p / SUB1;
                        cx<T>& dst = lines[pidx(p - (m1 - (m1 >> 1)) * SUB1)];
                        if (m1 & 1) dst.y = (T)Phi;
                        else dst.x = (T)Phi;
                    } else {
                        lines[pidx(p)] = mk<T>((T)Phi, 0);
                    }
                }
            } else {
                const int M = a.M;
                const TA eps = a.eps;
#pragma unroll
                for (int j = 0; j < PB; ++j) {
                    const int p = p0 + j * blockDim.x;
                    if (p >= NPX) break;
                    const TA ex = rd_sfc ? (TA)se[1][j] : slot(a.s_etax, p);
                    const TA ez = rd_sfc ? (TA)se[2][j] : slot(a.s_etaz, p);
                    const TA px = slot(a.s_psix, p), pz = slot(a.s_psiz, p);
                    const TA g0 = slot(a.s_g0psi, p);
                    const TA g2 = ex * ex + ez * ez;
                    const TA d = ex * px + ez * pz;
                    const TA q2 = px * px + pz * pz;
                    TA Gnl = 0;
                    if (M >= 2) {
                        const TA eta = rd_sfc ? (TA)se[0][j] : slot(a.s_eta, p);
                        TA W = 0, ep = 1;
#pragma unroll
                        for (int q = 1; q <= kMaxOrder; ++q) {
                            if (q > M) break;
                            W += ep * (TA)slot(a.s_F0 + (M - q), p);
                            ep = ep * eta * (TA)(1.0 / q);
                        }
                        Gnl = (TA)a.epsp[M - 1] * W - eps * d;
                        if (M >= 3) Gnl += prev[j] + (TA)a.epsp[2] * g2 * g0;
                    }
                    const TA den = (TA)1 + (TA)a.epsp[2] * g2;
                    const TA Wb = (g0 + Gnl + eps * d) / den;
                    const TA Np = eps * ((TA)-0.5 * q2 + (TA)0.5 * den * Wb * Wb);
                    lines[pidx(p)] = mk<T>((T)Gnl, (T)Np);
                }
            }
        }
        __syncthreads();

        // Phase C: forward DIT of line 0; blocks of up to three line groups run it as one
        // group of compile-time width, wider blocks with run-time strides; keep kx < nx/2.
        {
            cx<T>* o0 = out0 + (long long)zp * HX;
            auto fwd0 = [&](auto st) {
                if constexpr (ONEG) {
                    P::template dit_wide<TL, false, T>(lines, tw, threadIdx.x, -1, st);
                } else if constexpr (TL >= 32) {
                    constexpr int kBarC = 15;
                    const int ng = blockDim.x / TL;
                    if (ng == 3) {
                        P::template dit_wide<3 * TL, false, T>(lines, tw, threadIdx.x, kBarC, st);
                    } else if (ng == 2) {
                        P::template dit_wide<2 * TL, false, T>(lines, tw, threadIdx.x, kBarC, st);
                    } else if (ng == 1) {
                        P::template dit_wide<TL, false, T>(lines, tw, threadIdx.x, kBarC, st);
                    } else {
                        P::template dit_blk<false, T>(lines, tw, threadIdx.x, blockDim.x, st);
                    }
                } else {
                    P::template dit_blk<false, T>(lines, tw, threadIdx.x, blockDim.x, st);
                }
            };
            if constexpr (HALF_OK) {
                if (half) {
                    // Z = DFT_{N/2}(x[2n] + i x[2n+1]); X[k] = E[k] + w_N^k O[k] with
                    // E = (Z[k] + conj Z[N/2-k]) / 2 and O = (Z[k] - conj Z[N/2-k]) / 2i
                    using PH = IPlan<NPX / 2, V>;
                    constexpr int NH = NPX / 2;
                    auto sth = [&](int k, cx<T> v) { lines[pidx(k)] = v; };
                    if constexpr (ONEG) {
                        PH::template dit_wide<TL, false, T>(lines, a.twh, threadIdx.x, -1, sth);
                    } else {
                        constexpr int kBarC = 15;
                        if (blockDim.x == 2 * TL) PH::template dit_wide<2 * TL, false, T>(lines, a.twh, threadIdx.x, kBarC, sth);
                        else PH::template dit_blk<false, T>(lines, a.twh, threadIdx.x, blockDim.x, sth);
                    }
                    __syncthreads();
                    for (int k = threadIdx.x; k < HX; k += blockDim.x) {
                        const cx<T> A = lines[pidx(k)];
                        const cx<T> B = cconj(lines[pidx(k == 0 ? 0 : NH - k)]);
                        const cx<T> D = csub(A, B);
                        const cx<T> E = cscale(cadd(A, B), (T)0.5);
                        const cx<T> O = mk<T>((T)0.5 * D.y, (T)-0.5 * D.x);
                        o0[k] = cadd(E, cmul(__ldg(&a.twr[k]), O));
                    }
                }
            }
            if (a.kind == 0 && !(HALF_OK && half)) {
                fwd0([&](int k, cx<T> v) {
                    if (k < HX) o0[k] = v;
                });
            } else if (a.kind != 0) {
                fwd0([&](int k, cx<T> v) { lines[pidx(k)] = v; });
                __syncthreads();
                cx<T>* o1 = out1 + (long long)zp * HX;
                for (int k = threadIdx.x; k < HX; k += blockDim.x) {
                    const cx<T> X = lines[pidx(k)];
                    const cx<T> Y = cconj(lines[pidx(k == 0 ? 0 : NPX - k)]);
                    o0[k] = cscale(cadd(X, Y), (T)0.5);
                    const cx<T> D = csub(X, Y);
                    o1[k] = mk<T>((T)0.5 * D.y, (T)-0.5 * D.x);
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Column kernel: CB columns per block, tiles loaded and stored cooperatively.
// ---------------------------------------------------------------------------
// Per-column shared-memory stride (complex elements): rounded so that
// stride = 4 (mod 16), which puts the CB columns of 4 consecutive rows of a
// cooperative tile access on distinct 8-byte banks.
__host__ __device__ constexpr int col_stride(int need) { return (need + 15) / 16 * 16 + 4; }

// Dynamic shared memory of a column-kernel block with `groups` line groups: per
// column, the line and the truncated spectrum S (spectral kinds) or two lines (final).
template <typename T, int NPZ, int DIV>
__host__ __device__ constexpr size_t col_smem_bytes(bool final_kind, int groups) {
    return (size_t)groups * (final_kind ? col_stride(2 * line_stride(NPZ)) : col_stride(line_stride(NPZ) + 2 * NPZ / DIV)) *
           sizeof(cx<T>);
}

// Cooperative load of a [NR x CB] tile (rows 0..NR-1, columns c0..c0+CB-1 of a row-major
// [NR][hx] complex array; columns at or past hx read as zero) into shared memory at
// sm[cg * per + slot(z)]. Each thread issues all of its loads before its first store, so
// the tile costs about one memory round trip: the column kernels run one block per SM and
// nothing else hides this phase.
template <typename T, int NR, int CB, int NT, class Slot>
__device__ __forceinline__ void col2_load_tile(const cx<T>* __restrict__ src, int hx, int c0, cx<T>* sm, int per,
                                               Slot slot) {
    constexpr int N = NR * CB;
    constexpr int PERT = (N + NT - 1) / NT;
    cx<T> v[PERT];
#pragma unroll
    for (int j = 0; j < PERT; ++j) {
        const int i = threadIdx.x + j * NT;
        const int z = i / CB, cg = i - z * CB;
        v[j] = ((N % NT == 0 || i < N) && c0 + cg < hx) ? __ldg(src + (long long)z * hx + c0 + cg) : mk<T>(0, 0);
    }
#pragma unroll
    for (int j = 0; j < PERT; ++j) {
        const int i = threadIdx.x + j * NT;
        const int z = i / CB, cg = i - z * CB;
        if (N % NT == 0 || i < N) sm[(size_t)cg * per + slot(z)] = v[j];
    }
}

// The same tile through asynchronous global -> shared copies (cp.async, one element each), for
// the final pass's two tiles: with no register staging both are in flight at once and cost one
// memory round trip instead of two (that pass -3 %; the single-tile passes gained nothing from
// it). Columns at or past hx are zeroed with plain stores. The caller waits with
// cp_async_wait_all() before its block barrier.
template <typename T, int NR, int CB, int NT, class Slot>
__device__ __forceinline__ void col2_load_tile_async(const cx<T>* __restrict__ src, int hx, int c0, cx<T>* sm,
                                                     int per, Slot slot) {
    constexpr int N = NR * CB;
#pragma unroll 4
    for (int i = threadIdx.x; i < N; i += NT) {
        const int z = i / CB, cg = i - z * CB;
        cx<T>* d = sm + (size_t)cg * per + slot(z);
        if (c0 + cg < hx) {
            const unsigned sa = (unsigned)__cvta_generic_to_shared(d);
            asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(sa),
                         "l"(src + (long long)z * hx + c0 + cg), "n"((int)sizeof(cx<T>))
                         : "memory");
        } else {
            *d = mk<T>(0, 0);
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename T, int NPZ, int CB, int NT>
__device__ __forceinline__ void col2_store_tile(const cx<T>* sm, int per, cx<T>* dst, int c0, int hx) {
    constexpr int N = NPZ * CB;
#pragma unroll 4
    for (int i = threadIdx.x; i < N; i += NT) {
        const int z = i / CB, cg = i - z * CB;
        if (c0 + cg < hx) dst[(long long)z * hx + c0 + cg] = sm[(size_t)cg * per + pidx(z)];
    }
}

// The final pass's update of one kept mode (kx index col, kz index mz) at compact index idx:
// the right-hand side from the transformed nonlinear parts Fe, Fp (scaled and tapered; Fe is
// zero at k = 0) and the linear parts G0 psi_hat, -g eta_hat, then the mode's epilogue (RK4
// stage combination with the Eq. 17 filter at the last stage, IF-AB2 of Eqs. 15-16, IF-RK4,
// the right-hand side itself, the inverse DNO update of Eq. 19, or the FP64 energy sums).
template <typename T>
__device__ __forceinline__ void fin_mode(const ColArgs<T>& a, long long idx, int col, int mz, cx<T> Fe, cx<T> Fp,
                                         T hh, T ihx, T inz2, double& e_kin, double& e_pot, double& e_bad) {
    const T kxc = a.kx0 * (T)col;
    const T kz = a.kz0 * (T)mz;
    const T k = d_kabs(kxc * kxc + kz * kz);
    const cx<T> se = a.s_eta[idx], sp = a.s_psi[idx];
    const T G0 = k * tanh_kh(k * hh);
    cx<T> de = cadd(cscale(sp, G0), Fe);
    if (col == 0 && mz == 0) de = mk<T>(0, 0);
    const cx<T> dp = cadd(cscale(se, -a.g), Fp);
    switch (a.mode) {
    case FIN_INVDNO: {
        // Eq. 19: psi <- G0^{-1} (v - [G(eta) - G0] psi); the k = 0 mode keeps its value
        if (!(col == 0 && mz == 0)) a.y_psi[idx] = cscale(csub(a.v_hat[idx], Fe), (T)1 / G0);
    } break;
    case FIN_IFAB2: {
        // Eqs. 15-16: exact linear rotation plus the Duhamel response to the
        // AB2-extrapolated forcing F* (IF-Euler at the first step).
        cx<T> Fse = Fe, Fsp = Fp;
        if (!a.ab_first) {
            Fse = csub(cscale(Fe, (T)1.5), cscale(a.h_eta[idx], (T)0.5));
            Fsp = csub(cscale(Fp, (T)1.5), cscale(a.h_psi[idx], (T)0.5));
        }
        a.h_eta[idx] = Fe;
        a.h_psi[idx] = Fp;
        const T w = d_sqrt(a.g * G0);
        T c, sw, G0sw, gsw, omc_g, omc_G0;
        if (w > (T)0) {
            T sh, ch;                              // half angle: one sincos gives both
            d_sincos((T)0.5 * w * a.dt, &sh, &ch);
            const T omc = (T)2 * sh * sh;          // 1 - cos(w dt) without cancellation
            c = (T)1 - omc;
            sw = (T)2 * sh * ch / w;               // sin(w dt) / w
            G0sw = G0 * sw;                        // (G0 / w) sin(w dt)
            gsw = a.g * sw;                        // (g / w) sin(w dt)
            omc_g = omc / a.g;
            omc_G0 = omc / G0;
        } else {                                   // k = 0 limits stated under Eq. 16
            c = 1; sw = a.dt; G0sw = 0; gsw = a.g * a.dt; omc_g = 0; omc_G0 = (T)0.5 * a.g * a.dt * a.dt;
        }
        cx<T> e1 = cadd(cadd(cscale(se, c), cscale(sp, G0sw)), cadd(cscale(Fse, sw), cscale(Fsp, omc_g)));
        cx<T> p1 = cadd(csub(cscale(sp, c), cscale(se, gsw)), csub(cscale(Fsp, sw), cscale(Fse, omc_G0)));
        if (a.filter) {
            const T rx = (T)col * ihx;
            const T rz = (T)(mz < 0 ? -mz : mz) * inz2;
            const T A = (T)0.125 * ((T)5 + (T)4 * d_cospi(rx) - d_cospi((T)2 * rx)) *
                        ((T)0.125 * ((T)5 + (T)4 * d_cospi(rz) - d_cospi((T)2 * rz)));
            e1 = cscale(e1, A);
            p1 = cscale(p1, A);
        }
        a.y_eta[idx] = e1;
        a.y_psi[idx] = p1;
    } break;
    case FIN_RHS:
        a.ko_eta[idx] = de; a.ko_psi[idx] = dp;
        break;
    case FIN_IRK1:
    case FIN_IRK2:
    case FIN_IRK3:
    case FIN_IRK4: {
        // Integrating-factor RK4 (Lawson): the linear flow E_t of Eq. 14 exactly, RK4 on
        // the nonlinear part k = (Fe, Fp) of this stage in the rotating frame.
        const T w = d_sqrt(a.g * G0);
        T c1, s1, c2, s2;                          // cos and sin/w of w h/2 and of w h
        if (w > (T)0) {
            T sh, ch;
            d_sincos((T)0.5 * w * a.dt, &sh, &ch);
            c1 = ch; s1 = sh / w;
            c2 = (T)1 - (T)2 * sh * sh; s2 = (T)2 * sh * ch / w;
        } else {                                   // k = 0: E_t (e, p) = (e, p - g t e)
            c1 = 1; s1 = (T)0.5 * a.dt; c2 = 1; s2 = a.dt;
        }
        auto rot_e = [&](cx<T> e, cx<T> pp, T c, T sw) { return cadd(cscale(e, c), cscale(pp, G0 * sw)); };
        auto rot_p = [&](cx<T> e, cx<T> pp, T c, T sw) { return csub(cscale(pp, c), cscale(e, a.g * sw)); };
        const T hh = a.dt;
        const cx<T> ye = a.y_eta[idx], yp = a.y_psi[idx];
        if (a.mode == FIN_IRK1) {
            a.ka_eta[idx] = rot_e(Fe, Fp, c2, s2);
            a.ka_psi[idx] = rot_p(Fe, Fp, c2, s2);
            const cx<T> ue = cadd(ye, cscale(Fe, (T)0.5 * hh)), up = cadd(yp, cscale(Fp, (T)0.5 * hh));
            a.ys_eta[idx] = rot_e(ue, up, c1, s1);
            a.ys_psi[idx] = rot_p(ue, up, c1, s1);
        } else if (a.mode == FIN_IRK2) {
            a.ka_eta[idx] = cadd(a.ka_eta[idx], cscale(rot_e(Fe, Fp, c1, s1), (T)2));
            a.ka_psi[idx] = cadd(a.ka_psi[idx], cscale(rot_p(Fe, Fp, c1, s1), (T)2));
            a.ys_eta[idx] = cadd(rot_e(ye, yp, c1, s1), cscale(Fe, (T)0.5 * hh));
            a.ys_psi[idx] = cadd(rot_p(ye, yp, c1, s1), cscale(Fp, (T)0.5 * hh));
        } else if (a.mode == FIN_IRK3) {
            const cx<T> ke = rot_e(Fe, Fp, c1, s1), kp = rot_p(Fe, Fp, c1, s1);
            a.ka_eta[idx] = cadd(a.ka_eta[idx], cscale(ke, (T)2));
            a.ka_psi[idx] = cadd(a.ka_psi[idx], cscale(kp, (T)2));
            a.ys_eta[idx] = cadd(rot_e(ye, yp, c2, s2), cscale(ke, hh));
            a.ys_psi[idx] = cadd(rot_p(ye, yp, c2, s2), cscale(kp, hh));
        } else {
            T A = 1;
            if (a.filter) {
                const T rx = (T)col * ihx;
                const T rz = (T)(mz < 0 ? -mz : mz) * inz2;
                A = (T)0.125 * ((T)5 + (T)4 * d_cospi(rx) - d_cospi((T)2 * rx)) *
                    ((T)0.125 * ((T)5 + (T)4 * d_cospi(rz) - d_cospi((T)2 * rz)));
            }
            const T w6 = hh / (T)6;
            const cx<T> ne = cadd(rot_e(ye, yp, c2, s2), cscale(cadd(a.ka_eta[idx], Fe), w6));
            const cx<T> np = cadd(rot_p(ye, yp, c2, s2), cscale(cadd(a.ka_psi[idx], Fp), w6));
            a.y_eta[idx] = cscale(ne, A);
            a.y_psi[idx] = cscale(np, A);
        }
    } break;
    case FIN_RK1: {
        a.ka_eta[idx] = de; a.ka_psi[idx] = dp;
        const T hd = (T)0.5 * a.dt;
        a.ys_eta[idx] = cadd(a.y_eta[idx], cscale(de, hd));
        a.ys_psi[idx] = cadd(a.y_psi[idx], cscale(dp, hd));
    } break;
    case FIN_RK2:
    case FIN_RK3: {
        a.ka_eta[idx] = cadd(a.ka_eta[idx], cscale(de, (T)2));
        a.ka_psi[idx] = cadd(a.ka_psi[idx], cscale(dp, (T)2));
        const T hd = a.mode == FIN_RK2 ? (T)0.5 * a.dt : a.dt;
        a.ys_eta[idx] = cadd(a.y_eta[idx], cscale(de, hd));
        a.ys_psi[idx] = cadd(a.y_psi[idx], cscale(dp, hd));
    } break;
    case FIN_RK4: {
        const T w = a.dt / (T)6;
        T A = 1;
        if (a.filter) {
            const T rx = (T)col * ihx;
            const T rz = (T)(mz < 0 ? -mz : mz) * inz2;
            A = (T)0.125 * ((T)5 + (T)4 * d_cospi(rx) - d_cospi((T)2 * rx)) *
                ((T)0.125 * ((T)5 + (T)4 * d_cospi(rz) - d_cospi((T)2 * rz)));
        }
        const cx<T> ye = cadd(a.y_eta[idx], cscale(cadd(a.ka_eta[idx], de), w));
        const cx<T> yp = cadd(a.y_psi[idx], cscale(cadd(a.ka_psi[idx], dp), w));
        a.y_eta[idx] = cscale(ye, A);
        a.y_psi[idx] = cscale(yp, A);
    } break;
    case FIN_ENERGY: {
        const double wgt = col == 0 ? 1.0 : 2.0;
        e_kin += wgt * ((double)sp.x * (double)de.x + (double)sp.y * (double)de.y);
        e_pot += wgt * ((double)se.x * (double)se.x + (double)se.y * (double)se.y);
        const bool fin = isfinite((double)se.x) && isfinite((double)se.y) &&
                         isfinite((double)sp.x) && isfinite((double)sp.y);
        if (!fin) e_bad += 1.0;
    } break;
    default: break;
    }
}

// Where the final pass's two lines per column leave room for a single block per SM (over half
// of the SM's shared memory), say so to the compiler: it may then use the registers that
// occupancy leaves free instead of spilling. 0 leaves the minimum unspecified.
template <typename T, int NPZ, int CB>
constexpr int col_min_blocks() {
    return (size_t)CB * col_stride(2 * line_stride(NPZ)) * sizeof(cx<T>) > 116 * 1024 ? 1 : 0;
}

template <typename T, int NPZ, int CB, int V = 0, int DIV = 3>
__global__ void __launch_bounds__(CB * IPlan<NPZ, V>::TL < 32 ? 32 : CB * IPlan<NPZ, V>::TL,
                                  col_min_blocks<T, NPZ, CB>())
col2_kernel(const ColArgs<T> a, const cx<T>* __restrict__ tw) {
    using P = IPlan<NPZ, V>;
    constexpr int TL = P::TL;
    constexpr int NZ = 2 * NPZ / DIV;
    constexpr int LS = line_stride(NPZ);
    constexpr int NT = CB * TL < 32 ? 32 : CB * TL;   // threads of the block (the launch uses exactly this)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
    const int g = threadIdx.x / TL, lt = threadIdx.x % TL;
    const int bar = 1 + (g & 7);
    const int c0 = blockIdx.x * CB;
    const int c = c0 + g;
    const bool valid = (g < CB) && (c < a.hx);
    const int cc = valid ? c : c0;
    const T kx = a.kx0 * (T)cc;
    const long long oc = (long long)blockIdx.y * a.tcol;   // this tile's column-space fields
    const long long os = (long long)blockIdx.y * a.tst;    // this tile's compact spectra
    const T hh = a.hb ? a.hb[blockIdx.y] : a.h;
    const T ikc2 = (T)1 / (a.kc * a.kc);                   // taper argument |k|^2 / kc^2
    const T ihx = (T)1 / (T)a.hx, inz2 = (T)1 / (T)(NZ / 2);  // filter arguments |k_a| / kNyq_a

    if (a.kind == COL_FROM_STATE || a.kind == COL_PHI) {
        constexpr int PER = col_stride(LS + NZ);
        cx<T>* line = sm + (size_t)g * PER;
        cx<T>* S = line + LS;
        const int nsrc = a.kind == COL_FROM_STATE ? 2 : 1;
        for (int src = 0; src < nsrc; ++src) {
            if (a.kind == COL_FROM_STATE) {
                const cx<T>* st = (src == 0 ? a.st_eta : a.st_psi) + os;
                col2_load_tile<T, NZ, CB, NT>(st, a.hx, c0, sm, PER, [](int z) { return LS + z; });
                __syncthreads();
            } else {
                col2_load_tile<T, NPZ, CB, NT>(a.pin + oc, a.hx, c0, sm, PER, [](int z) { return pidx(z); });
                __syncthreads();
                // forward DIT: truncate to the kept modes, scale and taper into S
                const T fs = a.fscale;
                P::template dit<false, T>(line, tw, lt, bar, [&](int k, cx<T> v) {
                    int mz;
                    if (k < NZ / 2) mz = k;
                    else if (k > NPZ - NZ / 2) mz = k - NPZ;
                    else return;
                    const T kz = a.kz0 * (T)mz;
                    T s = fs;
                    if (a.taper) s *= d_taper((kx * kx + kz * kz) * ikc2);
                    S[mz >= 0 ? mz : mz + NZ] = cscale(v, s);
                });
                if (lt == 0) S[NZ / 2] = mk<T>(0, 0);
                __syncthreads();
            }
            for (int o = 0; o < a.nout; ++o) {
                if (a.out_src[o] != src) continue;
                const int sym = a.out_sym[o], aa = a.out_a[o];
                const T isc = a.iscale;
                constexpr int SUB1 = NPZ / P::R1;
                auto ld = [&](int ip, int ms) -> cx<T> {
                    int mz;
                    if (ms + SUB1 <= NZ / 2) mz = ip;
                    else if (ms >= NZ / 2 && ms + SUB1 <= NPZ - NZ / 2 + 1) return mk<T>(0, 0);
                    else if (ms > NPZ - NZ / 2) mz = ip - NPZ;
                    else if (ip < NZ / 2) mz = ip;
                    else if (ip > NPZ - NZ / 2) mz = ip - NPZ;
                    else return mk<T>(0, 0);
                    const int iz = mz >= 0 ? mz : mz + NZ;
                    const cx<T> s = S[iz];
                    const T kz = a.kz0 * (T)mz;
                    if (sym == SYM_ID) return cscale(s, isc);
                    if (sym == SYM_DZ) return cscale(mk<T>(-kz * s.y, kz * s.x), isc);
                    const T k2 = kx * kx + kz * kz;
                    T f = isc;
                    // |k|^(2 floor(a/2)), a <= kMaxOrder: predicated products, no per-element loop
                    const int e2 = aa >> 1;
#pragma unroll
                    for (int i = 0; i < kMaxOrder / 2; ++i)
                        if (i < e2) f *= k2;
                    if (aa & 1) {                                  // odd a: one more G0 = |k| tanh(|k| h)
                        const T k = d_kabs(k2);
                        f *= k * tanh_kh(k * hh);
                    }
                    return cscale(s, f);
                };
                P::template dif<true, T>(line, tw, lt, bar, ld);
                __syncthreads();
                col2_store_tile<T, NPZ, CB, NT>(sm, PER, a.colbase + oc + (long long)a.out_f[o] * a.fstride, c0, a.hx);
                __syncthreads();
            }
        }
        return;
    }

    // COL_FINAL: two products, forward DIT, linear parts, epilogue per natural mode
    constexpr int PER = col_stride(2 * LS);
    cx<T>* l0 = sm + (size_t)g * PER;
    cx<T>* l1 = l0 + LS;
    // The epilogue's state rows were written by the previous stage long before and come from
    // DRAM: request this tile's rows into L2 now, so that the fetch overlaps the tile load and
    // the two transforms (one prefetch per 32-byte sector, the addresses the epilogue reads).
    // Grids below 1024 points per axis keep their state in L2: no prefetch there.
    if (NPZ >= 1536 && !a.split) {
        const cx<T>* pf[6] = {a.s_eta, a.s_psi, nullptr, nullptr, nullptr, nullptr};
        int npf = 2;
        if (a.mode >= FIN_RK1 && a.mode <= FIN_RK4) {
            pf[npf++] = a.y_eta;
            pf[npf++] = a.y_psi;
            if (a.mode != FIN_RK1) { pf[npf++] = a.ka_eta; pf[npf++] = a.ka_psi; }
        }
        constexpr int PER_SECTOR = 32 / (int)sizeof(cx<T>) > 0 ? 32 / (int)sizeof(cx<T>) : 1;
        for (int i = threadIdx.x; i < NZ * npf; i += blockDim.x) {
            const int q = i / NZ, ic = i - q * NZ;
            const cx<T>* row = pf[q] + os + (long long)ic * a.hx + c0;
            for (int cg = 0; cg < CB && c0 + cg < a.hx; cg += PER_SECTOR)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(row + cg));
        }
    }
    col2_load_tile_async<T, NPZ, CB, NT>(a.gin + oc, a.hx, c0, sm, PER, [](int z) { return pidx(z); });
    col2_load_tile_async<T, NPZ, CB, NT>(a.nin + oc, a.hx, c0, sm, PER, [](int z) { return LS + pidx(z); });
    cp_async_wait_all();
    __syncthreads();
    P::template dit<false, T>(l0, tw, lt, bar, [&](int k, cx<T> v) { l0[pidx(k)] = v; });
    P::template dit<false, T>(l1, tw, lt, bar, [&](int k, cx<T> v) { l1[pidx(k)] = v; });
    __syncthreads();

    // Epilogue over the CB-column tile: consecutive threads take adjacent
    // columns of one kz row, so the state arrays move in 8*CB-byte segments.
    double e_kin = 0.0, e_pot = 0.0, e_bad = 0.0;
    for (int i = threadIdx.x; i < NZ * CB; i += blockDim.x) {
        const int ic = i / CB, cg = i - ic * CB;
        const int col = c0 + cg;
        if (col >= a.hx) continue;
        const long long idx = os + (long long)ic * a.hx + col;
        if (ic == NZ / 2) {
            if (a.mode == FIN_RHS && !a.split) { a.ko_eta[idx] = mk<T>(0, 0); a.ko_psi[idx] = mk<T>(0, 0); }
            continue;
        }
        const int mz = ic < NZ / 2 ? ic : ic - NZ;
        const int ip = mz >= 0 ? mz : mz + NPZ;
        const T kxc = a.kx0 * (T)col;
        const T kz = a.kz0 * (T)mz;
        T s = a.fscale;
        if (a.taper) s *= d_taper((kxc * kxc + kz * kz) * ikc2);
        const cx<T>* lc = sm + (size_t)cg * PER;
        cx<T> Fe = cscale(lc[pidx(ip)], s);
        const cx<T> Fp = cscale(lc[LS + pidx(ip)], s);
        if (col == 0 && mz == 0) Fe = mk<T>(0, 0);   // d eta/dt has zero mean
        if (a.split) {
            // the update runs in fin_epilogue_kernel, over the compact spectra
            a.fe[idx] = Fe;
            a.fp[idx] = Fp;
            continue;
        }
        fin_mode(a, idx, col, mz, Fe, Fp, hh, ihx, inz2, e_kin, e_pot, e_bad);
    }
    if (a.mode == FIN_ENERGY) {
        __shared__ double red[3][16];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            e_kin += __shfl_down_sync(0xffffffffu, e_kin, o);
            e_pot += __shfl_down_sync(0xffffffffu, e_pot, o);
            e_bad += __shfl_down_sync(0xffffffffu, e_bad, o);
        }
        const int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) { red[0][w] = e_kin; red[1][w] = e_pot; red[2][w] = e_bad; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double s0 = 0, s1 = 0, s2 = 0;
            for (int t = 0; t < (int)(blockDim.x >> 5); ++t) { s0 += red[0][t]; s1 += red[1][t]; s2 += red[2][t]; }
            const long long pb = 3 * ((long long)blockIdx.y * gridDim.x + blockIdx.x);
            a.partial[pb + 0] = s0;
            a.partial[pb + 1] = s1;
            a.partial[pb + 2] = s2;
        }
    }
}



// The final pass's update as its own launch over the compact spectra (consecutive threads
// take consecutive kx of one kz row): the column kernel then ends with its transforms and the
// update, which waits on the stage state in global memory, runs with every warp of the SM.
// Same arithmetic as the fused epilogue of col2_kernel. Not for FIN_ENERGY (block partials).
template <typename T>
__global__ void __launch_bounds__(256) fin_epilogue_kernel(const ColArgs<T> a) {
    const int nz = a.nz_grid;
    const long long n = (long long)nz * a.hx;
    const long long os = (long long)blockIdx.y * a.tst;
    const T hh = a.hb ? a.hb[blockIdx.y] : a.h;
    const T ihx = (T)1 / (T)a.hx, inz2 = (T)1 / (T)(nz / 2);
    double e_kin = 0.0, e_pot = 0.0, e_bad = 0.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int ic = (int)(e / a.hx), col = (int)(e - (long long)ic * a.hx);
        const long long idx = os + e;
        if (ic == nz / 2) {
            if (a.mode == FIN_RHS) { a.ko_eta[idx] = mk<T>(0, 0); a.ko_psi[idx] = mk<T>(0, 0); }
            continue;
        }
        const int mz = ic < nz / 2 ? ic : ic - nz;
        fin_mode(a, idx, col, mz, a.fe[idx], a.fp[idx], hh, ihx, inz2, e_kin, e_pot, e_bad);
    }
}

// ---------------------------------------------------------------------------
// Learned closure: features in, residual out (compact spectra [nz][hx]).
// ---------------------------------------------------------------------------
struct ClosureScales { float in[6]; float out[2]; };

// Six feature spectra at state (se, sp) with the low-order right-hand side
// (de, dp): eta, i kx eta, i kz eta, G0 psi, de - G0 psi, dp + g eta, each
// divided by its input scale; the z Nyquist row is zero.
template <typename T>
__global__ void closure_prep_kernel(const cx<T>* __restrict__ se, const cx<T>* __restrict__ sp,
                                    const cx<T>* __restrict__ de, const cx<T>* __restrict__ dp, cx<T>* __restrict__ out,
                                    int nz, int hx, T kx0, T kz0, T h, T g, ClosureScales sc) {
    const long long n = (long long)nz * hx;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int ic = (int)(i / hx), col = (int)(i - (long long)ic * hx);
        cx<T> v[6];
        if (ic == nz / 2) {
            for (int c = 0; c < 6; ++c) v[c] = mk<T>(0, 0);
        } else {
            const int mz = ic < nz / 2 ? ic : ic - nz;
            const T kx = kx0 * (T)col, kz = kz0 * (T)mz;
            const T k = d_sqrt(kx * kx + kz * kz);
            const T G0 = k * tanh_kh(k * h);
            const cx<T> e = se[i], p = sp[i];
            const cx<T> g0p = cscale(p, G0);
            v[0] = e;
            v[1] = mk<T>(-kx * e.y, kx * e.x);
            v[2] = mk<T>(-kz * e.y, kz * e.x);
            v[3] = g0p;
            v[4] = csub(de[i], g0p);
            v[5] = cadd(dp[i], cscale(e, g));
        }
        for (int c = 0; c < 6; ++c) out[(long long)c * n + i] = cscale(v[c], (T)(1.0f / sc.in[c]));
    }
}

// Corrected right-hand side (ko + out_scale T(k) R_hat, eta's k = 0 mode zero)
// followed by the same epilogue as the final column kernel: FIN_RHS writes it
// back to ko, FIN_RK1..4 combine the RK4 stages (filter of Eq. 17 at the last).
template <typename T>
__global__ void closure_combine_kernel(ColArgs<T> a, const cx<T>* __restrict__ Re, const cx<T>* __restrict__ Rp,
                                       ClosureScales sc) {
    const int NZ = a.nz_grid, hx = a.hx;
    const long long n = (long long)NZ * hx;
    const T ihx = (T)1 / (T)hx, inz2 = (T)1 / (T)(NZ / 2);
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int ic = (int)(idx / hx), col = (int)(idx - (long long)ic * hx);
        if (ic == NZ / 2) {
            if (a.mode == FIN_RHS) { a.ko_eta[idx] = mk<T>(0, 0); a.ko_psi[idx] = mk<T>(0, 0); }
            continue;
        }
        const int mz = ic < NZ / 2 ? ic : ic - NZ;
        const T kxc = a.kx0 * (T)col, kz = a.kz0 * (T)mz;
        T tp = 1;
        if (a.taper) {
            const T kk2 = (kxc * kxc + kz * kz) / (a.kc * a.kc);
            const T k4 = kk2 * kk2;
            tp = d_exp(-(k4 * k4));
        }
        cx<T> de = cadd(a.ko_eta[idx], cscale(Re[idx], (T)sc.out[0] * tp));
        const cx<T> dp = cadd(a.ko_psi[idx], cscale(Rp[idx], (T)sc.out[1] * tp));
        if (col == 0 && mz == 0) de = mk<T>(0, 0);
        switch (a.mode) {
        case FIN_RHS:
            a.ko_eta[idx] = de; a.ko_psi[idx] = dp;
            break;
        case FIN_RK1: {
            a.ka_eta[idx] = de; a.ka_psi[idx] = dp;
            const T hd = (T)0.5 * a.dt;
            a.ys_eta[idx] = cadd(a.y_eta[idx], cscale(de, hd));
            a.ys_psi[idx] = cadd(a.y_psi[idx], cscale(dp, hd));
        } break;
        case FIN_RK2:
        case FIN_RK3: {
            a.ka_eta[idx] = cadd(a.ka_eta[idx], cscale(de, (T)2));
            a.ka_psi[idx] = cadd(a.ka_psi[idx], cscale(dp, (T)2));
            const T hd = a.mode == FIN_RK2 ? (T)0.5 * a.dt : a.dt;
            a.ys_eta[idx] = cadd(a.y_eta[idx], cscale(de, hd));
            a.ys_psi[idx] = cadd(a.y_psi[idx], cscale(dp, hd));
        } break;
        case FIN_RK4: {
            const T w = a.dt / (T)6;
            T A = 1;
            if (a.filter) {
                const T rx = (T)col * ihx;
                const T rz = (T)(mz < 0 ? -mz : mz) * inz2;
                A = (T)0.125 * ((T)5 + (T)4 * d_cospi(rx) - d_cospi((T)2 * rx)) *
                    ((T)0.125 * ((T)5 + (T)4 * d_cospi(rz) - d_cospi((T)2 * rz)));
            }
            const cx<T> ye = cadd(a.y_eta[idx], cscale(cadd(a.ka_eta[idx], de), w));
            const cx<T> yp = cadd(a.y_psi[idx], cscale(cadd(a.ka_psi[idx], dp), w));
            a.y_eta[idx] = cscale(ye, A);
            a.y_psi[idx] = cscale(yp, A);
        } break;
        default: break;
        }
    }
}

// out_c = (hi_c - lo_c) / scale_c for the two components (compact spectra).
template <typename T>
__global__ void closure_diff_kernel(const cx<T>* __restrict__ hi, const cx<T>* __restrict__ lo, cx<T>* __restrict__ out,
                                    long long n, ClosureScales sc) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < 2 * n; i += (long long)gridDim.x * blockDim.x)
        out[i] = cscale(csub(hi[i], lo[i]), (T)(1.0f / sc.out[i < n ? 0 : 1]));
}

// Adaptive order: FP64 sums over the half spectrum (kx > 0 columns weighted 2)
// of |lo - hi|^2 and |hi|^2, both components, into part[2 * block].
template <typename T>
__global__ void diff_norm_kernel(const cx<T>* __restrict__ he, const cx<T>* __restrict__ hp,
                                 const cx<T>* __restrict__ le, const cx<T>* __restrict__ lp, int nz, int hx,
                                 double* __restrict__ part) {
    const long long n = (long long)nz * hx;
    double num = 0.0, den = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int col = (int)(i % hx);
        const double w = col == 0 ? 1.0 : 2.0;
        const cx<T> a = he[i], b = hp[i], c = le[i], d = lp[i];
        const double ex = (double)c.x - a.x, ey = (double)c.y - a.y, px = (double)d.x - b.x, py = (double)d.y - b.y;
        num += w * (ex * ex + ey * ey + px * px + py * py);
        den += w * ((double)a.x * a.x + (double)a.y * a.y + (double)b.x * b.x + (double)b.y * b.y);
    }
    __shared__ double red[2][32];
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_down_sync(0xffffffffu, num, o);
        den += __shfl_down_sync(0xffffffffu, den, o);
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = num; red[1][threadIdx.x >> 5] = den; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { x += red[0][w]; y += red[1][w]; }
        part[2 * blockIdx.x] = x;
        part[2 * blockIdx.x + 1] = y;
    }
}

// Fallback check: with D = f_high - f_low (d = 6 .. 1 / 2) and the predicted
// P = out_scale T(k) R_hat, FP64 sums of |D - P|^2 and |D|^2 over the half
// spectrum (kx > 0 columns weighted 2) into part[2 * block].
template <typename T>
__global__ void closure_err_kernel(const cx<T>* __restrict__ fe, const cx<T>* __restrict__ fp,
                                   const cx<T>* __restrict__ le, const cx<T>* __restrict__ lp,
                                   const cx<T>* __restrict__ Re, const cx<T>* __restrict__ Rp, int nz, int hx, T kx0,
                                   T kz0, T kc, int taper, ClosureScales sc, double* __restrict__ part) {
    const long long n = (long long)nz * hx;
    double num = 0.0, den = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int ic = (int)(i / hx), col = (int)(i - (long long)ic * hx);
        if (ic == nz / 2) continue;
        const int mz = ic < nz / 2 ? ic : ic - nz;
        const T kx = kx0 * (T)col, kz = kz0 * (T)mz;
        T tp = 1;
        if (taper) {
            const T kk2 = (kx * kx + kz * kz) / (kc * kc);
            const T k4 = kk2 * kk2;
            tp = d_exp(-(k4 * k4));
        }
        const double w = col == 0 ? 1.0 : 2.0;
        const bool zero = col == 0 && mz == 0;
        const cx<T> De = csub(fe[i], le[i]), Dp = csub(fp[i], lp[i]);
        const cx<T> Pe = zero ? mk<T>(0, 0) : cscale(Re[i], (T)sc.out[0] * tp);
        const cx<T> Pp = cscale(Rp[i], (T)sc.out[1] * tp);
        const double ex = (double)De.x - Pe.x, ey = (double)De.y - Pe.y;
        const double px = (double)Dp.x - Pp.x, py = (double)Dp.y - Pp.y;
        num += w * (ex * ex + ey * ey + px * px + py * py);
        den += w * ((double)De.x * De.x + (double)De.y * De.y + (double)Dp.x * Dp.x + (double)Dp.y * Dp.y);
    }
    __shared__ double red[2][32];
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_down_sync(0xffffffffu, num, o);
        den += __shfl_down_sync(0xffffffffu, den, o);
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = num; red[1][threadIdx.x >> 5] = den; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += red[0][w]; b += red[1][w]; }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

}  // namespace zk
