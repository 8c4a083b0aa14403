// zk_kernels.cuh - the kernels of one Zakharov right-hand side and its stages.
//
// Data flow of one right-hand-side evaluation at order M (Sec. 3.2, Sec. 6.1).
// Spectra are stored as half spectra along x: a "compact" field is
// [nz][nx/2] complex (kz rows in FFT order, kx = 0 .. nx/2-1; the x Nyquist
// column is not stored, the z Nyquist row is held at zero). A "column-space"
// field is [npz][nx/2] complex: z already transformed to the 3/2-padded
// physical grid (npz = 3 nz / 2), x still spectral. Padded physical fields
// ([npz][npx]) reach global memory only as the series accumulator and the
// three surface planes eta, dx eta, dz eta (written by round 1, read by the
// later rounds instead of transforming the same three fields again).
//
// The launches of one right-hand side (kernels in zk_kernels2.cuh):
//  col2_kernel COL_FROM_STATE: per kx column, read the stage state
//      eta_hat, psi_hat and write column-space eta, dz eta, psi, dz psi and
//      dz^a psi for a = 1..M (zero padding, inverse column FFT).
//  row2_kernel round r = 1..M-1: per padded row, inverse row FFTs of
//      F_j = dz^{r-j} Phi(j) (j < r) into physical space (round 1 also
//      transforms eta, dx eta, dz eta and writes the surface planes; later
//      rounds read them); pointwise Phi(r) = -sum eta^{r-j}/(r-j)! F_j and
//      W(r-1) = sum eta^{r-1-j}/(r-1-j)! F_j; W(r-1) folded into the series
//      accumulator with its eps and |grad eta|^2 weights; forward row FFT of
//      Phi(r) into column space.
//  col2_kernel COL_PHI (round r): forward column FFT of Phi(r), truncate to
//      the kept modes, taper -> Phi_hat(r); write dz^a Phi(r), a = 1..M-r.
//  row2_kernel final round M: W(M-1), the full G_nl = sum eps^m G_m,
//      W of Eq. 11 and the Bernoulli term of Eq. 10; forward row FFT of the
//      pair (G_nl, N_psi).
//  col2_kernel COL_FINAL: forward column FFTs, truncate, taper, add the
//      linear parts G0 psi_hat and -g eta_hat, zero the mean of d eta/dt, then
//      the epilogue: RK4 stage combination (+ state filter of Eq. 17 at the
//      last stage), IF-AB2 update, output of the right-hand side, the inverse
//      DNO fixed-point update or the FP64 energy partials.
// This file holds their argument blocks and the unpadded state I/O, tank and
// relaxation kernels.
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
    // batched tiles (blockIdx.y = tile): element offsets of one tile's
    // column-space fields and of its accumulator; 0 for a single grid
    long long tcol, tacc;
    int nb;                  // tiles in the launch (host side: grid.y)
    int occ;                 // host side: resident blocks per SM to use (0 = all)
    int acc64;               // host side: series sums in FP64 (FP32 contexts; acc holds doubles)
    int pad3;                // host side: 3N padding (kernels with DIV = 6)
    // Surface planes: eta, d eta/dx, d eta/dz on the padded grid, [3][npz][npx] (positions in
    // the row plan's digit-reversed order). sfc_mode 0: not used (the round transforms them
    // from their slots); 1: the round transforms them and writes the planes; 2: the round
    // reads them from the planes and has no slots for them. tsfc: one tile's element offset.
    T* sfc;
    long long tsfc;
    int sfc_mode;
    // Half-length forward transform of the real Phi(r) (intermediate rounds): the table of the
    // N/2 plan and w_N^k = exp(-2 pi i k / N) for k < N/2; nullptr = full-length transform.
    const cx<T>* twh;
    const cx<T>* twr;
};

// ---------------------------------------------------------------------------
// Column side
// ---------------------------------------------------------------------------
enum ColKind { COL_FROM_STATE = 0, COL_PHI = 1, COL_FINAL = 2 };
enum ColSym { SYM_ID = 0, SYM_DZ = 1, SYM_ZA = 2 };
enum FinalMode { FIN_RHS = 0, FIN_RK1 = 1, FIN_RK2 = 2, FIN_RK3 = 3, FIN_RK4 = 4, FIN_ENERGY = 5, FIN_IFAB2 = 6,
                 FIN_INVDNO = 7, FIN_IRK1 = 8, FIN_IRK2 = 9, FIN_IRK3 = 10, FIN_IRK4 = 11 };

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
    // batched tiles (blockIdx.y = tile): element offsets of one tile's
    // column-space fields and of its compact spectra, per-tile depth h
    long long tcol, tst;
    const T* hb;                    // nullptr: every tile has depth h
    int nb;                         // tiles in the launch (host side: grid.y)
    int pad3;                       // host side: 3N padding (kernels with DIV = 6)
    // kind 2: split = 1 stores the transformed nonlinear parts (Fe, Fp) to fe / fp (compact)
    // and leaves the update to fin_epilogue_kernel
    int split;
    cx<T>* fe;
    cx<T>* fp;
};

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

// cols: in-place column transforms of two compact fields [nz][hx] (forward sets the z Nyquist
// row to zero). A block takes CB adjacent columns: the tiles move as [nz][CB] row segments
// (consecutive threads on adjacent columns of one row, so every 32-byte sector is used whole),
// each column is transformed in shared memory by its own group of TL threads. Column slots are
// PER apart, with PER mod 16 chosen so that a half-warp's 64-bit tile accesses hit distinct banks.
template <int NZ>
__host__ __device__ constexpr int cols_cb() {
    return Plan<NZ>::TL >= 32 ? 4 : 128 / Plan<NZ>::TL;
}
template <int NZ>
__host__ __device__ constexpr int cols_per() {
    return (line_stride(NZ) + 15) / 16 * 16 + (cols_cb<NZ>() >= 16 ? 1 : 16 / cols_cb<NZ>());
}
template <typename T, int NZ>
__host__ __device__ constexpr size_t cols_smem_bytes() {
    return (size_t)cols_cb<NZ>() * cols_per<NZ>() * sizeof(cx<T>);
}

template <typename T, int NZ, bool INV>
__global__ void cols_kernel(cx<T>* f0, cx<T>* f1, int hx, const cx<T>* __restrict__ tw) {
    using P = Plan<NZ>;
    constexpr int TL = P::TL;
    constexpr int CB = cols_cb<NZ>();
    constexpr int PER = cols_per<NZ>();
    constexpr int NT = CB * TL;                    // the launch uses exactly this block size
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
    const int g = threadIdx.x / TL, lt = threadIdx.x % TL;
    const int bar = 1 + (g & 7);
    cx<T>* line = sm + (size_t)g * PER;
    const int c0 = blockIdx.x * CB;
    for (int f = 0; f < 2; ++f) {
        cx<T>* fp = f == 0 ? f0 : f1;
        if (!fp) continue;
        // the z Nyquist row is zero by convention; an inverse never reads it
        for (int i = threadIdx.x; i < NZ * CB; i += NT) {
            const int z = i / CB, cg = i - z * CB, col = c0 + cg;
            sm[(size_t)cg * PER + pidx(z)] =
                (col < hx && !(INV && z == NZ / 2)) ? fp[(long long)z * hx + col] : mk<T>(0, 0);
        }
        __syncthreads();
        P::template run<INV, T>(line, tw, lt, bar);
        __syncthreads();
        for (int i = threadIdx.x; i < NZ * CB; i += NT) {
            const int z = i / CB, cg = i - z * CB, col = c0 + cg;
            if (col < hx) {
                cx<T> v = sm[(size_t)cg * PER + pidx(z)];
                if (!INV && z == NZ / 2) v = mk<T>(0, 0);
                fp[(long long)z * hx + col] = v;
            }
        }
        __syncthreads();
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
