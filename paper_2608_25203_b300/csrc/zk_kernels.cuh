// zk_kernels.cuh - the kernels of one Zakharov right-hand side and its stages.
//
// Data flow of one right-hand-side evaluation at order M (Sec. 3.2, Sec. 6.1).
// Spectra are stored as half spectra along x: a "compact" field is
// [nz][nx/2] complex (kz rows in FFT order, kx = 0 .. nx/2-1; the x Nyquist
// column is not stored, the z Nyquist row is held at zero). A "column-space"
// field is [npz][nx/2] complex: z already transformed to the 3/2-padded
// physical grid (npz = 3 nz / 2), x still spectral. Padded physical fields
// ([npz][npx]) never reach global memory except the series accumulator.
//
//  col_kernel kind 0 (round 0): per kx column, read the stage state
//      eta_hat, psi_hat and write column-space eta, dz eta, psi, dz psi and
//      dz^a psi for a = 1..M (zero padding, inverse column FFT).
//  row_round_kernel round r = 1..M-1: per padded row, inverse row FFTs of
//      eta, [dx eta, dz eta], F_j = dz^{r-j} Phi(j) (j < r) into physical
//      space; pointwise Phi(r) = -sum eta^{r-j}/(r-j)! F_j and
//      W(r-1) = sum eta^{r-1-j}/(r-1-j)! F_j; W(r-1) folded into the series
//      accumulator with its eps and |grad eta|^2 weights; forward row FFT of
//      Phi(r) into column space.
//  col_kernel kind 1 (round r): forward column FFT of Phi(r), truncate to
//      the kept modes, taper -> Phi_hat(r); write dz^a Phi(r), a = 1..M-r.
//  row_round_kernel final round M: W(M-1), the full G_nl = sum eps^m G_m,
//      W of Eq. 11 and the Bernoulli term of Eq. 10; forward row FFT of the
//      pair (G_nl, N_psi).
//  col_kernel kind 2: forward column FFTs, truncate, taper, add the linear
//      parts G0 psi_hat and -g eta_hat, zero the mean of d eta/dt, then the
//      epilogue: RK4 stage combination (+ state filter of Eq. 17 at the last
//      stage), output of the right-hand side, or the FP64 energy partials.
#pragma once

#include "zk_fft.cuh"

namespace zk {

constexpr int kMaxOrder = 8;
constexpr int kMaxLines = 8;
constexpr int kMaxColOut = 16;

template <typename T> __device__ __forceinline__ T d_tanh(T x);
template <> __device__ __forceinline__ float d_tanh<float>(float x) { return tanhf(x); }
template <> __device__ __forceinline__ double d_tanh<double>(double x) { return tanh(x); }
template <typename T> __device__ __forceinline__ T d_exp(T x);
template <> __device__ __forceinline__ float d_exp<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double d_exp<double>(double x) { return exp(x); }
template <typename T> __device__ __forceinline__ T d_sqrt(T x);
template <> __device__ __forceinline__ float d_sqrt<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double d_sqrt<double>(double x) { return sqrt(x); }
template <typename T> __device__ __forceinline__ T d_cospi(T x);
template <> __device__ __forceinline__ float d_cospi<float>(float x) { return cospif(x); }
template <> __device__ __forceinline__ double d_cospi<double>(double x) { return cospi(x); }

// ---------------------------------------------------------------------------
// Row side
// ---------------------------------------------------------------------------
template <typename T>
struct RowArgs {
    const cx<T>* colbase;    // column-space field f at colbase + f * fstride
    long long fstride;       // npz * hx
    int nlines;              // complex lines (two real fields each)
    int fa[kMaxLines], fb[kMaxLines];   // field index of re / im component, -1 = none
    unsigned dxa, dxb;       // bit l: multiply component by i kx before the inverse transform
    int kind;                // 0 = intermediate round r, 1 = final round (r = M)
    int r, M;
    int s_eta, s_etax, s_etaz, s_psix, s_psiz, s_g0psi, s_F0;   // slot of each physical field
    T eps;
    T epsp[kMaxOrder + 3];   // eps^j
    T kx0;                   // 2 pi / Lx
    T* acc;                  // [npz][npx] series accumulator
    cx<T>* out0;             // column-space output (Phi(r), or G_nl)
    cx<T>* out1;             // N_psi (final round)
    int npz;                 // padded rows (persistent row kernels loop over them)
};

template <typename T, int NPX>
__global__ void __launch_bounds__(512) row_round_kernel(const RowArgs<T> a, const cx<T>* __restrict__ tw) {
    using P = Plan<NPX>;
    constexpr int TL = P::TL;
    constexpr int HX = NPX / 3;
    constexpr int LS = line_stride(NPX);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* lines = reinterpret_cast<cx<T>*>(smem_raw);
    const int zp = blockIdx.x;
    const int g = threadIdx.x / TL, lt = threadIdx.x % TL;
    const int bar = 1 + (g & 7);
    cx<T>* buf = lines + (size_t)g * LS;
    const int ngroups = blockDim.x / TL;

    // Phase A: Hermitian-packed spectrum of two real fields, inverse row FFT.
    if (g < a.nlines) {
        const int fa = a.fa[g], fb = a.fb[g];
        const bool da = (a.dxa >> g) & 1u, db = (a.dxb >> g) & 1u;
        const cx<T>* pa = fa >= 0 ? a.colbase + (long long)fa * a.fstride + (long long)zp * HX : nullptr;
        const cx<T>* pb = fb >= 0 ? a.colbase + (long long)fb * a.fstride + (long long)zp * HX : nullptr;
        for (int m = lt; m < NPX; m += TL) {
            int mm = -1;
            bool mir = false;
            if (m < HX) mm = m;
            else if (m > NPX - HX) { mm = NPX - m; mir = true; }
            cx<T> z = mk<T>(0, 0);
            if (mm >= 0) {
                cx<T> A = pa ? pa[mm] : mk<T>(0, 0);
                cx<T> B = pb ? pb[mm] : mk<T>(0, 0);
                const T kx = a.kx0 * (T)mm;
                if (da) A = mk<T>(-kx * A.y, kx * A.x);
                if (db) B = mk<T>(-kx * B.y, kx * B.x);
                if (mm == 0) { A.y = 0; B.y = 0; }
                z = mir ? mk<T>(A.x + B.y, B.x - A.y) : mk<T>(A.x - B.y, A.y + B.x);
            }
            buf[pidx(m)] = z;
        }
    } else {
        for (int m = lt; m < NPX; m += TL) buf[pidx(m)] = mk<T>(0, 0);
    }
    group_sync<TL>(bar);
    P::template run<true, T>(buf, tw, lt, bar);
    __syncthreads();

    // Phase B: pointwise HOS terms on the padded row.
    auto slot = [&](int s, int p) -> T {
        const cx<T> v = lines[(s >> 1) * LS + pidx(p)];
        return (s & 1) ? v.y : v.x;
    };
    T* accrow = a.acc + (long long)zp * NPX;
    for (int p = threadIdx.x; p < NPX; p += blockDim.x) {
        if (a.kind == 0) {
            const int r = a.r;
            const T eta = slot(a.s_eta, p);
            T W = 0, Phi = 0, ep = 1;
            for (int q = 1; q <= r; ++q) {
                const T eq = ep * eta / (T)q;
                const T F = slot(a.s_F0 + (r - q), p);
                W += ep * F;
                Phi -= eq * F;
                ep = eq;
            }
            if (r >= 2) {
                T coef = a.epsp[r - 1];
                if (r - 1 <= a.M - 3) {
                    const T ex = slot(a.s_etax, p), ez = slot(a.s_etaz, p);
                    coef += a.epsp[r + 1] * (ex * ex + ez * ez);
                }
                const T prev = (r == 2) ? (T)0 : accrow[p];
                accrow[p] = prev + coef * W;
            }
            lines[pidx(p)] = mk<T>(Phi, 0);
        } else {
            const int M = a.M;
            const T eps = a.eps;
            const T ex = slot(a.s_etax, p), ez = slot(a.s_etaz, p);
            const T px = slot(a.s_psix, p), pz = slot(a.s_psiz, p);
            const T g0 = slot(a.s_g0psi, p);
            const T g2 = ex * ex + ez * ez;
            const T d = ex * px + ez * pz;
            const T q2 = px * px + pz * pz;
            T Gnl = 0;
            if (M >= 2) {
                const T eta = slot(a.s_eta, p);
                T W = 0, ep = 1;
                for (int q = 1; q <= M; ++q) {
                    W += ep * slot(a.s_F0 + (M - q), p);
                    ep = ep * eta / (T)q;
                }
                Gnl = a.epsp[M - 1] * W - eps * d;
                if (M >= 3) Gnl += accrow[p] + a.epsp[2] * g2 * g0;
            }
            const T den = (T)1 + a.epsp[2] * g2;
            const T Wb = (g0 + Gnl + eps * d) / den;
            const T Np = eps * ((T)-0.5 * q2 + (T)0.5 * den * Wb * Wb);
            lines[pidx(p)] = mk<T>(Gnl, Np);
        }
    }
    __syncthreads();

    // Phase C: forward row FFT of the output line, keep kx < nx/2.
    if (threadIdx.x < 32 || g == 0) {
        P::template run<false, T>(lines + (size_t)g * LS, tw, lt, bar);
    }
    if (g == 0) {
        cx<T>* o0 = a.out0 + (long long)zp * HX;
        if (a.kind == 0) {
            for (int k = lt; k < HX; k += TL) o0[k] = lines[pidx(k)];
        } else {
            cx<T>* o1 = a.out1 + (long long)zp * HX;
            for (int k = lt; k < HX; k += TL) {
                const cx<T> X = lines[pidx(k)];
                const cx<T> Y = cconj(lines[pidx(k == 0 ? 0 : NPX - k)]);
                o0[k] = cscale(cadd(X, Y), (T)0.5);
                const cx<T> D = csub(X, Y);
                o1[k] = mk<T>((T)0.5 * D.y, (T)-0.5 * D.x);   // -(i/2) D
            }
        }
    }
    (void)ngroups;
}

// ---------------------------------------------------------------------------
// Column side
// ---------------------------------------------------------------------------
enum ColKind { COL_FROM_STATE = 0, COL_PHI = 1, COL_FINAL = 2 };
enum ColSym { SYM_ID = 0, SYM_DZ = 1, SYM_ZA = 2 };
enum FinalMode { FIN_RHS = 0, FIN_RK1 = 1, FIN_RK2 = 2, FIN_RK3 = 3, FIN_RK4 = 4, FIN_ENERGY = 5, FIN_IFAB2 = 6,
                 FIN_INVDNO = 7 };

template <typename T>
struct ColArgs {
    int kind, hx, nz_grid;
    T kx0, kz0, h, g, kc;
    int taper;
    T fscale;                 // (nx nz)/(npx npz): truncation back to the kept modes
    T iscale;                 // 1/(nx nz): into padded physical values
    const cx<T>* st_eta;      // kind 0: compact [nz][hx]
    const cx<T>* st_psi;
    const cx<T>* pin;         // kind 1: column-space Phi(r)
    cx<T>* colbase;
    long long fstride;
    int nout;
    int out_f[kMaxColOut], out_src[kMaxColOut], out_sym[kMaxColOut], out_a[kMaxColOut];
    // kind 2
    const cx<T>* gin;
    const cx<T>* nin;
    int mode;
    const cx<T>* s_eta;       // state the right-hand side is evaluated at
    const cx<T>* s_psi;
    cx<T>* y_eta; cx<T>* y_psi;     // step-start state (updated at the last RK stage)
    cx<T>* ys_eta; cx<T>* ys_psi;   // next stage state
    cx<T>* ka_eta; cx<T>* ka_psi;   // RK accumulator
    cx<T>* ko_eta; cx<T>* ko_psi;   // right-hand side output
    T dt;
    int filter;
    int nx_grid;
    double* partial;          // energy: [gridDim.x][3]
    cx<T>* h_eta; cx<T>* h_psi;     // IF-AB2: nonlinear forcing of the previous step
    const cx<T>* v_hat;             // inverse DNO: target v = G(eta) psi (compact)
    int ab_first;                   // IF-AB2: 1 = bootstrap with IF-Euler (F* = F_n)
};

template <typename T>
__device__ __forceinline__ T za_symbol(T k, T G0, int a) {
    // dz^a of a flat-strip harmonic mode: |k|^a (a even), |k|^(a-1) G0 (a odd)
    T p = 1;
    const int e = (a & 1) ? a - 1 : a;
    for (int i = 0; i < e; ++i) p *= k;
    return (a & 1) ? p * G0 : p;
}

template <typename T, int NPZ>
__device__ __forceinline__ void col_fill_and_store(const ColArgs<T>& a, const cx<T>* S, cx<T>* line,
                                                   int c, int lt, int bar, int src, const cx<T>* __restrict__ tw) {
    using P = Plan<NPZ>;
    constexpr int TL = P::TL;
    constexpr int NZ = 2 * NPZ / 3;
    const T kx = a.kx0 * (T)c;
    for (int o = 0; o < a.nout; ++o) {
        if (a.out_src[o] != src) continue;
        const int sym = a.out_sym[o], aa = a.out_a[o];
        for (int ip = lt; ip < NPZ; ip += TL) {
            int mz = 0;
            bool keep = true;
            if (ip < NZ / 2) mz = ip;
            else if (ip > NPZ - NZ / 2) mz = ip - NPZ;
            else keep = false;
            cx<T> v = mk<T>(0, 0);
            if (keep) {
                const int ic = mz >= 0 ? mz : mz + NZ;
                const cx<T> s = S[ic];
                const T kz = a.kz0 * (T)mz;
                if (sym == SYM_ID) {
                    v = cscale(s, a.iscale);
                } else if (sym == SYM_DZ) {
                    v = cscale(mk<T>(-kz * s.y, kz * s.x), a.iscale);
                } else {
                    const T k = d_sqrt(kx * kx + kz * kz);
                    const T G0 = k * d_tanh(k * a.h);
                    v = cscale(s, za_symbol(k, G0, aa) * a.iscale);
                }
            }
            line[pidx(ip)] = v;
        }
        group_sync<TL>(bar);
        P::template run<true, T>(line, tw, lt, bar);
        cx<T>* dst = a.colbase + (long long)a.out_f[o] * a.fstride + c;
        for (int z = lt; z < NPZ; z += TL) dst[(long long)z * a.hx] = line[pidx(z)];
        group_sync<TL>(bar);
    }
}

template <typename T, int NPZ, int CB>
__global__ void __launch_bounds__(CB * Plan<NPZ>::TL < 32 ? 32 : CB * Plan<NPZ>::TL)
col_kernel(const ColArgs<T> a, const cx<T>* __restrict__ tw) {
    using P = Plan<NPZ>;
    constexpr int TL = P::TL;
    constexpr int NZ = 2 * NPZ / 3;
    constexpr int LS = line_stride(NPZ);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
    const int g = threadIdx.x / TL, lt = threadIdx.x % TL;
    const int bar = 1 + (g & 7);
    const int c = blockIdx.x * CB + g;
    const bool valid = (g < CB) && (c < a.hx);
    const int cc = valid ? c : 0;   // inactive groups run on column 0 and store nothing

    if (a.kind == COL_FROM_STATE || a.kind == COL_PHI) {
        cx<T>* line = sm + (size_t)g * (LS + NZ);
        cx<T>* S = line + LS;
        if (a.kind == COL_FROM_STATE) {
            for (int src = 0; src < 2; ++src) {
                const cx<T>* st = src == 0 ? a.st_eta : a.st_psi;
                for (int i = lt; i < NZ; i += TL) S[i] = st[(long long)i * a.hx + cc];
                group_sync<TL>(bar);
                if (valid) {
                    col_fill_and_store<T, NPZ>(a, S, line, cc, lt, bar, src, tw);
                } else {
                    // keep warp-level synchronisation uniform for narrow groups
                    ColArgs<T> dummy = a;
                    (void)dummy;
                    for (int o = 0; o < a.nout; ++o) {
                        if (a.out_src[o] != src) continue;
                        group_sync<TL>(bar);
                        P::template run<true, T>(line, tw, lt, bar);
                        group_sync<TL>(bar);
                    }
                }
                group_sync<TL>(bar);
            }
        } else {
            for (int z = lt; z < NPZ; z += TL) line[pidx(z)] = a.pin[(long long)z * a.hx + cc];
            group_sync<TL>(bar);
            P::template run<false, T>(line, tw, lt, bar);
            const T kx = a.kx0 * (T)cc;
            for (int ic = lt; ic < NZ; ic += TL) {
                cx<T> v = mk<T>(0, 0);
                if (ic != NZ / 2) {
                    const int mz = ic < NZ / 2 ? ic : ic - NZ;
                    const int ip = mz >= 0 ? mz : mz + NPZ;
                    const T kz = a.kz0 * (T)mz;
                    T s = a.fscale;
                    if (a.taper) {
                        const T k = d_sqrt(kx * kx + kz * kz) / a.kc;
                        const T k2 = k * k, k4 = k2 * k2;
                        s *= d_exp(-(k4 * k4));
                    }
                    v = cscale(line[pidx(ip)], s);
                }
                S[ic] = v;
            }
            group_sync<TL>(bar);
            if (valid) {
                col_fill_and_store<T, NPZ>(a, S, line, cc, lt, bar, 0, tw);
            } else {
                for (int o = 0; o < a.nout; ++o) {
                    group_sync<TL>(bar);
                    P::template run<true, T>(line, tw, lt, bar);
                    group_sync<TL>(bar);
                }
            }
        }
        return;
    }

    // COL_FINAL
    cx<T>* l0 = sm + (size_t)g * (2 * LS);
    cx<T>* l1 = l0 + LS;
    for (int z = lt; z < NPZ; z += TL) {
        l0[pidx(z)] = a.gin[(long long)z * a.hx + cc];
        l1[pidx(z)] = a.nin[(long long)z * a.hx + cc];
    }
    group_sync<TL>(bar);
    P::template run<false, T>(l0, tw, lt, bar);
    P::template run<false, T>(l1, tw, lt, bar);

    double e_kin = 0.0, e_pot = 0.0, e_bad = 0.0;
    if (valid) {
        const T kx = a.kx0 * (T)cc;
        const T ax = a.filter && a.mode == FIN_RK4
                         ? (T)0.125 * ((T)5 + (T)4 * d_cospi((T)cc / (T)a.hx) - d_cospi((T)2 * (T)cc / (T)a.hx))
                         : (T)1;
        for (int ic = lt; ic < NZ; ic += TL) {
            if (ic == NZ / 2) {
                if (a.mode == FIN_RHS) {
                    const long long idx = (long long)ic * a.hx + cc;
                    a.ko_eta[idx] = mk<T>(0, 0);
                    a.ko_psi[idx] = mk<T>(0, 0);
                }
                continue;
            }
            const int mz = ic < NZ / 2 ? ic : ic - NZ;
            const int ip = mz >= 0 ? mz : mz + NPZ;
            const T kz = a.kz0 * (T)mz;
            const T k = d_sqrt(kx * kx + kz * kz);
            T s = a.fscale;
            if (a.taper) {
                const T kk = k / a.kc;
                const T k2 = kk * kk, k4 = k2 * k2;
                s *= d_exp(-(k4 * k4));
            }
            cx<T> Fe = cscale(l0[pidx(ip)], s);
            const cx<T> Fp = cscale(l1[pidx(ip)], s);
            if (cc == 0 && mz == 0) Fe = mk<T>(0, 0);   // d eta/dt has zero mean
            const long long idx = (long long)ic * a.hx + cc;
            const cx<T> se = a.s_eta[idx], sp = a.s_psi[idx];
            const T G0 = k * d_tanh(k * a.h);
            cx<T> de = cadd(cscale(sp, G0), Fe);
            if (cc == 0 && mz == 0) de = mk<T>(0, 0);
            const cx<T> dp = cadd(cscale(se, -a.g), Fp);
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
                T A = ax;
                if (a.filter) {
                    const T rz = (T)(mz < 0 ? -mz : mz) / (T)(NZ / 2);
                    A *= (T)0.125 * ((T)5 + (T)4 * d_cospi(rz) - d_cospi((T)2 * rz));
                }
                const cx<T> ye = cadd(a.y_eta[idx], cscale(cadd(a.ka_eta[idx], de), w));
                const cx<T> yp = cadd(a.y_psi[idx], cscale(cadd(a.ka_psi[idx], dp), w));
                a.y_eta[idx] = cscale(ye, A);
                a.y_psi[idx] = cscale(yp, A);
            } break;
            case FIN_ENERGY: {
                const double wgt = cc == 0 ? 1.0 : 2.0;
                e_kin += wgt * ((double)sp.x * (double)de.x + (double)sp.y * (double)de.y);
                e_pot += wgt * ((double)se.x * (double)se.x + (double)se.y * (double)se.y);
                const bool fin = isfinite((double)se.x) && isfinite((double)se.y) &&
                                 isfinite((double)sp.x) && isfinite((double)sp.y);
                if (!fin) e_bad += 1.0;
            } break;
            default: break;
            }
        }
    }
    if (a.mode == FIN_ENERGY) {
        // fixed-order FP64 reduction: shuffle tree per warp, then warps in order
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
            a.partial[3 * blockIdx.x + 0] = s0;
            a.partial[3 * blockIdx.x + 1] = s1;
            a.partial[3 * blockIdx.x + 2] = s2;
        }
    }
}

static __global__ void energy_finalize_kernel(const double* __restrict__ partial, int n, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s0 = 0, s1 = 0, s2 = 0;
        for (int i = 0; i < n; ++i) { s0 += partial[3 * i]; s1 += partial[3 * i + 1]; s2 += partial[3 * i + 2]; }
        out[0] = s0; out[1] = s1; out[2] = s2;
    }
}

// ---------------------------------------------------------------------------
// Unpadded transforms for state input / output
// ---------------------------------------------------------------------------
// rows_fwd: physical rows of two real fields -> half spectra [nz][nx/2] (kx < nx/2)
template <typename T, typename TIN, int NX>
__global__ void rows_fwd_kernel(const TIN* __restrict__ fa, const TIN* __restrict__ fb, int nz,
                                cx<T>* __restrict__ oa, cx<T>* __restrict__ ob, const cx<T>* __restrict__ tw) {
    using P = Plan<NX>;
    constexpr int TL = P::TL;
    constexpr int LS = line_stride(NX);
    constexpr int HX = NX / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = threadIdx.x / TL, lt = threadIdx.x % TL;
    const int bar = 1 + (g & 7);
    cx<T>* line = reinterpret_cast<cx<T>*>(smem_raw) + (size_t)g * LS;
    const int z = blockIdx.x * (blockDim.x / TL) + g;
    const bool valid = z < nz;
    const int zz = valid ? z : 0;
    for (int p = lt; p < NX; p += TL)
        line[pidx(p)] = mk<T>((T)fa[(long long)zz * NX + p], (T)fb[(long long)zz * NX + p]);
    group_sync<TL>(bar);
    P::template run<false, T>(line, tw, lt, bar);
    if (valid) {
        for (int k = lt; k < HX; k += TL) {
            const cx<T> X = line[pidx(k)];
            const cx<T> Y = cconj(line[pidx(k == 0 ? 0 : NX - k)]);
            oa[(long long)z * HX + k] = cscale(cadd(X, Y), (T)0.5);
            const cx<T> D = csub(X, Y);
            ob[(long long)z * HX + k] = mk<T>((T)0.5 * D.y, (T)-0.5 * D.x);
        }
    }
}

// rows_inv: two half spectra [nz][nx/2] -> physical rows, scaled by `scale`
template <typename T, typename TOUT, int NX>
__global__ void rows_inv_kernel(const cx<T>* __restrict__ ia, const cx<T>* __restrict__ ib, int nz, T scale,
                                TOUT* __restrict__ fa, TOUT* __restrict__ fb, const cx<T>* __restrict__ tw) {
    using P = Plan<NX>;
    constexpr int TL = P::TL;
    constexpr int LS = line_stride(NX);
    constexpr int HX = NX / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = threadIdx.x / TL, lt = threadIdx.x % TL;
    const int bar = 1 + (g & 7);
    cx<T>* line = reinterpret_cast<cx<T>*>(smem_raw) + (size_t)g * LS;
    const int z = blockIdx.x * (blockDim.x / TL) + g;
    const bool valid = z < nz;
    const int zz = valid ? z : 0;
    for (int m = lt; m < NX; m += TL) {
        int mm = -1;
        bool mir = false;
        if (m < HX) mm = m;
        else if (m > NX - HX) { mm = NX - m; mir = true; }
        cx<T> v = mk<T>(0, 0);
        if (mm >= 0) {
            cx<T> A = ia[(long long)zz * HX + mm];
            cx<T> B = ib ? ib[(long long)zz * HX + mm] : mk<T>(0, 0);
            if (mm == 0) { A.y = 0; B.y = 0; }
            v = mir ? mk<T>(A.x + B.y, B.x - A.y) : mk<T>(A.x - B.y, A.y + B.x);
        }
        line[pidx(m)] = v;
    }
    group_sync<TL>(bar);
    P::template run<true, T>(line, tw, lt, bar);
    if (valid) {
        for (int p = lt; p < NX; p += TL) {
            const cx<T> v = line[pidx(p)];
            fa[(long long)z * NX + p] = (TOUT)(v.x * scale);
            if (fb) fb[(long long)z * NX + p] = (TOUT)(v.y * scale);
        }
    }
}

// cols: in-place column transforms of `nf` compact fields [nz][hx] (forward
// sets the z Nyquist row to zero).
template <typename T, int NZ, bool INV>
__global__ void cols_kernel(cx<T>* f0, cx<T>* f1, int hx, const cx<T>* __restrict__ tw) {
    using P = Plan<NZ>;
    constexpr int TL = P::TL;
    constexpr int LS = line_stride(NZ);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = threadIdx.x / TL, lt = threadIdx.x % TL;
    const int bar = 1 + (g & 7);
    cx<T>* line = reinterpret_cast<cx<T>*>(smem_raw) + (size_t)g * LS;
    const int c = blockIdx.x * (blockDim.x / TL) + g;
    const bool valid = c < hx;
    const int cc = valid ? c : 0;
    for (int f = 0; f < 2; ++f) {
        cx<T>* fp = f == 0 ? f0 : f1;
        if (!fp) continue;
        // the z Nyquist row is zero by convention; an inverse never reads it
        for (int i = lt; i < NZ; i += TL)
            line[pidx(i)] = (INV && i == NZ / 2) ? mk<T>(0, 0) : fp[(long long)i * hx + cc];
        group_sync<TL>(bar);
        P::template run<INV, T>(line, tw, lt, bar);
        if (valid) {
            for (int i = lt; i < NZ; i += TL) {
                cx<T> v = line[pidx(i)];
                if (!INV && i == NZ / 2) v = mk<T>(0, 0);
                fp[(long long)i * hx + c] = v;
            }
        }
        group_sync<TL>(bar);
    }
}


// psi_hat = v_hat / G0 on every mode but k = 0 (first iterate of Eq. 19); the z
// Nyquist row is set to zero, the k = 0 mode of psi is left as it is.
template <typename T>
__global__ void inv_g0_kernel(const cx<T>* __restrict__ v, cx<T>* __restrict__ psi, int nz, int hx,
                              T kx0, T kz0, T h) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nz * hx) return;
    const int ic = i / hx, col = i - ic * hx;
    if (ic == nz / 2) { psi[i] = mk<T>(0, 0); return; }
    if (ic == 0 && col == 0) return;
    const int mz = ic < nz / 2 ? ic : ic - nz;
    const T kx = kx0 * (T)col, kz = kz0 * (T)mz;
    const T k = d_sqrt(kx * kx + kz * kz);
    const T G0 = k * d_tanh(k * h);
    psi[i] = cscale(v[i], (T)1 / G0);
}

// One row of a compact field (after its inverse column transform): inverse row
// FFT to the physical row, eta <- eta_t + (eta - eta_t) exp(-sigma dt)
// (Eq. 34), forward row FFT back to the half spectrum, in place.
template <typename T, typename TIN, int NX>
__global__ void relax_rows_kernel(cx<T>* __restrict__ f, const TIN* __restrict__ sigma,
                                  const TIN* __restrict__ target, int nz, T dt, T scale,
                                  const cx<T>* __restrict__ tw) {
    using P = Plan<NX>;
    constexpr int TL = P::TL;
    constexpr int LS = line_stride(NX);
    constexpr int HX = NX / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = threadIdx.x / TL, lt = threadIdx.x % TL;
    const int bar = 1 + (g & 7);
    cx<T>* line = reinterpret_cast<cx<T>*>(smem_raw) + (size_t)g * LS;
    const int z = blockIdx.x * (blockDim.x / TL) + g;
    const bool valid = z < nz;
    const int zz = valid ? z : 0;
    for (int m = lt; m < NX; m += TL) {
        int mm = -1;
        bool mir = false;
        if (m < HX) mm = m;
        else if (m > NX - HX) { mm = NX - m; mir = true; }
        cx<T> v = mk<T>(0, 0);
        if (mm >= 0) {
            cx<T> A = f[(long long)zz * HX + mm];
            if (mm == 0) A.y = 0;
            v = mir ? cconj(A) : A;
        }
        line[pidx(m)] = v;
    }
    group_sync<TL>(bar);
    P::template run<true, T>(line, tw, lt, bar);
    for (int p = lt; p < NX; p += TL) {
        const long long gi = (long long)zz * NX + p;
        const T e = line[pidx(p)].x * scale;
        const T t = (T)target[gi];
        const T r = t + (e - t) * d_exp(-(T)sigma[gi] * dt);
        line[pidx(p)] = mk<T>(r, 0);
    }
    group_sync<TL>(bar);
    P::template run<false, T>(line, tw, lt, bar);
    if (valid)
        for (int k = lt; k < HX; k += TL) f[(long long)z * HX + k] = line[pidx(k)];
}


// Even extension across reflecting walls (Sec. 3.3, Eq. 12): a tank field of
// mx x mz cell-centred samples becomes the (2mx) x (2mz) periodic field
// f~(i, k) = f(r(i), r(k)) with r(i) = i for i < m, 2m - 1 - i otherwise.
template <typename TIN>
__global__ void even_extend_kernel(const TIN* __restrict__ src, TIN* __restrict__ dst, int mx, int mz) {
    const int nx = 2 * mx;
    const long long n = (long long)nx * 2 * mz;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(t / nx), i = (int)(t - (long long)k * nx);
        const int si = i < mx ? i : nx - 1 - i;
        const int sk = k < mz ? k : 2 * mz - 1 - k;
        dst[t] = src[(long long)sk * mx + si];
    }
}

// The (0:mz, 0:mx) corner of a (2mx) x (2mz) field.
template <typename TIN>
__global__ void crop_kernel(const TIN* __restrict__ src, TIN* __restrict__ dst, int mx, int mz) {
    const long long n = (long long)mx * mz;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(t / mx), i = (int)(t - (long long)k * mx);
        dst[t] = src[(long long)k * 2 * mx + i];
    }
}

}  // namespace zk
