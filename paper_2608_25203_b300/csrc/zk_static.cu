// zk_static.cu - zk_dno_static: G(eta) psi with no device allocation.
//
// Some callers cannot call cudaMalloc: code embedded in a host application
// that owns the device memory pool (a raw cudaMalloc bypasses the pool's
// accounting, or fails once the pool has reserved the memory), and loops
// with latency limits that forbid allocation after start-up (cudaMalloc may
// synchronise the device and takes unbounded time). For them this file keeps
// every intermediate of one DNO evaluation in a fixed array in device memory,
// reserved when the library's device code is loaded, and the caller passes
// only the input and output arrays.
//
// The scratch array is shared by every call on a device and keeps the last
// call's contents; each call overwrites or clears everything it reads before
// reading it. Calls whose GPU work overlaps (different streams, or different
// host threads, on the same device) race on the array.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include <cuda.h>

#include "../../include/zk.h"
#include "zk_kernels2.cuh"

using namespace zk;

// Every GPU that loads this library holds this array until the process exits.
static __device__ __align__(256) unsigned char zk_static_scratch[ZK_STATIC_SCRATCH_BYTES];

namespace {

// Host code cannot use the array's name as a device address: the address is
// looked up with cudaGetSymbolAddress in the calling thread's current context
// and cached under that context's unique id (cuCtxGetId; ids are never reused
// within a process). A cudaDeviceReset, or a caller that makes another driver
// context current on the same device, therefore gets a fresh lookup instead of
// an address from a context that no longer holds the array. Where the driver
// entry points cannot be resolved, every call looks the address up.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
constexpr int kMaxContexts = 64;
std::mutex g_mu;
bool g_resolved = false;
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
unsigned long long g_ids[kMaxContexts] = {};
void* g_addr[kMaxContexts] = {};
int g_n = 0, g_next = 0;

void resolve_driver_entry_points() {
    if (g_resolved) return;
    g_resolved = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        g_ctx_id = reinterpret_cast<CtxGetIdFn>(f);
    cudaGetLastError();
}

// Unique id of the current context; false if there is none or it cannot be read.
bool current_context_id(unsigned long long* id) {
    if (!g_ctx_current || !g_ctx_id) return false;
    CUcontext ctx = nullptr;
    if (g_ctx_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return false;
    return g_ctx_id(ctx, id) == CUDA_SUCCESS;
}

zk_status lookup_symbol(void** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, zk_static_scratch);
    if (e != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return ZK_ECUDA;
    }
    *out = p;
    return ZK_OK;
}

zk_status scratch_address(void** out) {
    std::lock_guard<std::mutex> lk(g_mu);
    resolve_driver_entry_points();
    unsigned long long id = 0;
    if (current_context_id(&id)) {
        for (int i = 0; i < g_n; ++i)
            if (g_ids[i] == id) { *out = g_addr[i]; return ZK_OK; }
    }
    // first call in this context (the lookup also makes the runtime's context current)
    void* p = nullptr;
    const zk_status st = lookup_symbol(&p);
    if (st != ZK_OK) return st;
    if (current_context_id(&id)) {
        const int slot = g_n < kMaxContexts ? g_n++ : (g_next++ % kMaxContexts);
        g_ids[slot] = id;
        g_addr[slot] = p;
    }
    *out = p;
    return ZK_OK;
}

// w_n^t = exp(-2 pi i t / n) in FP64 on the device, rounded to FP32.
__global__ void static_twiddle_kernel(cx<float>* tw, int n) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) {
        double s, c;
        sincospi(-2.0 * (double)t / (double)n, &s, &c);
        tw[t] = mk<float>((float)c, (float)s);
    }
}

// Per-stage table of an in-place plan (entry e = w_B^{n1 m}), FP64 on the device.
__global__ void static_plan_twiddle_kernel(cx<float>* tw, PlanDesc d, int ne) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < ne) {
        long long num;
        int den;
        plan_table_entry(d, e, &num, &den);
        double s, c;
        sincospi(-2.0 * (double)num / (double)den, &s, &c);
        tw[e] = mk<float>((float)c, (float)s);
    }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

int field_count(int M) { return 4 + M + M * (M - 1) / 2 + 3; }

// Column-space field indices (same layout as a context uses).
struct SFields {
    int M;
    int base(int j) const { int b = 4 + M; for (int r = 1; r < j; ++r) b += M - r; return b; }
    int z(int j, int a) const { return j == 0 ? 3 + a : base(j) + a - 1; }
    int phiout() const { return base(M); }
    int gnl() const { return phiout() + 1; }
    int npsi() const { return phiout() + 2; }
};

struct Layout {
    size_t tw_x, tw_z, tw_px, tw_pz, y_eta, y_psi, ko_eta, ko_psi, col, acc, total;
};

Layout layout(int nx, int nz, int M) {
    const int npx = 3 * nx / 2, npz = 3 * nz / 2, hx = nx / 2;
    const size_t c = sizeof(cx<float>);
    Layout L;
    size_t o = 0;
    L.tw_x = o; o += align256((size_t)nx * c);
    L.tw_z = o; o += align256((size_t)nz * c);
    L.tw_px = o; o += align256((size_t)npx * c);
    L.tw_pz = o; o += align256((size_t)npz * c);
    const size_t comp = align256((size_t)nz * hx * c);
    L.y_eta = o; o += comp;
    L.y_psi = o; o += comp;
    L.ko_eta = o; o += comp;
    L.ko_psi = o; o += comp;
    L.col = o; o += align256((size_t)field_count(M) * npz * hx * c);
    L.acc = o; o += align256((size_t)npz * npx * sizeof(float));
    L.total = o;
    return L;
}

cudaError_t smem_attr(const void* fn, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int NPX>
cudaError_t s_row(const RowArgs<float>& a, const cx<float>* tw, int npz, cudaStream_t s) {
    constexpr int TL = IPlan<NPX>::TL;
    int nl = a.nlines, groups;
    if constexpr (TL < 32) { constexpr int per = 32 / TL; nl = (nl + per - 1) / per * per; groups = nl; }
    else groups = std::min(nl, kRowMaxThreads / TL);
    const size_t smem = (size_t)nl * line_stride(NPX) * sizeof(cx<float>);
    cudaError_t e = smem_attr((const void*)row2_kernel<float, NPX>, smem);
    if (e != cudaSuccess) return e;
    RowArgs<float> b = a;
    b.npz = npz;
    row2_kernel<float, NPX><<<npz, groups * TL, smem, s>>>(b, tw);
    return cudaGetLastError();
}
cudaError_t s_row_any(int npx, const RowArgs<float>& a, const cx<float>* tw, int npz, cudaStream_t s) {
    switch (npx) {
    case 24: return s_row<24>(a, tw, npz, s);
    case 48: return s_row<48>(a, tw, npz, s);
    case 96: return s_row<96>(a, tw, npz, s);
    case 192: return s_row<192>(a, tw, npz, s);
    case 384: return s_row<384>(a, tw, npz, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int NPZ>
cudaError_t s_col(const ColArgs<float>& a, const cx<float>* tw, cudaStream_t s) {
    constexpr int TL = IPlan<NPZ>::TL;
    constexpr int CB = TL >= 64 ? 4 : (128 / TL);
    constexpr int NZ = 2 * NPZ / 3;
    constexpr int LS = line_stride(NPZ);
    const int threads = CB * TL < 32 ? 32 : CB * TL;
    const size_t smem = col_smem_bytes<float, NPZ, 3>(a.kind == COL_FINAL, threads / TL);
    cudaError_t e = smem_attr((const void*)col2_kernel<float, NPZ, CB>, smem);
    if (e != cudaSuccess) return e;
    col2_kernel<float, NPZ, CB><<<(a.hx + CB - 1) / CB, threads, smem, s>>>(a, tw);
    return cudaGetLastError();
}
cudaError_t s_col_any(int npz, const ColArgs<float>& a, const cx<float>* tw, cudaStream_t s) {
    switch (npz) {
    case 24: return s_col<24>(a, tw, s);
    case 48: return s_col<48>(a, tw, s);
    case 96: return s_col<96>(a, tw, s);
    case 192: return s_col<192>(a, tw, s);
    case 384: return s_col<384>(a, tw, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int N>
cudaError_t s_rows_fwd(const float* fa, const float* fb, int nz, cx<float>* oa, cx<float>* ob, const cx<float>* tw, cudaStream_t s) {
    constexpr int TL = Plan<N>::TL;
    const int threads = TL >= 128 ? TL : 128, rows = threads / TL;
    const size_t smem = (size_t)rows * line_stride(N) * sizeof(cx<float>);
    cudaError_t e = smem_attr((const void*)rows_fwd_kernel<float, float, N>, smem);
    if (e != cudaSuccess) return e;
    rows_fwd_kernel<float, float, N><<<(nz + rows - 1) / rows, threads, smem, s>>>(fa, fb, nz, oa, ob, tw);
    return cudaGetLastError();
}
template <int N>
cudaError_t s_rows_inv(const cx<float>* ia, int nz, float scale, float* fa, const cx<float>* tw, cudaStream_t s) {
    constexpr int TL = Plan<N>::TL;
    const int threads = TL >= 128 ? TL : 128, rows = threads / TL;
    const size_t smem = (size_t)rows * line_stride(N) * sizeof(cx<float>);
    cudaError_t e = smem_attr((const void*)rows_inv_kernel<float, float, N>, smem);
    if (e != cudaSuccess) return e;
    rows_inv_kernel<float, float, N><<<(nz + rows - 1) / rows, threads, smem, s>>>(ia, nullptr, nz, scale, fa, nullptr, tw);
    return cudaGetLastError();
}
template <int N, bool INV>
cudaError_t s_cols(cx<float>* f0, cx<float>* f1, int hx, const cx<float>* tw, cudaStream_t s) {
    constexpr int CB = cols_cb<N>(), threads = CB * Plan<N>::TL;
    constexpr size_t smem = cols_smem_bytes<float, N>();
    cudaError_t e = smem_attr((const void*)cols_kernel<float, N, INV>, smem);
    if (e != cudaSuccess) return e;
    cols_kernel<float, N, INV><<<(hx + CB - 1) / CB, threads, smem, s>>>(f0, f1, hx, tw);
    return cudaGetLastError();
}

#define ZK_STATIC_SWITCH(n, CALL)                          \
    switch (n) {                                           \
    case 16: { constexpr int N_ = 16; return CALL; }       \
    case 32: { constexpr int N_ = 32; return CALL; }       \
    case 64: { constexpr int N_ = 64; return CALL; }       \
    case 128: { constexpr int N_ = 128; return CALL; }     \
    case 256: { constexpr int N_ = 256; return CALL; }     \
    default: return cudaErrorInvalidValue;                 \
    }

cudaError_t rows_fwd_any(int nx, const float* fa, const float* fb, int nz, cx<float>* oa, cx<float>* ob, const cx<float>* tw, cudaStream_t s) {
    ZK_STATIC_SWITCH(nx, (s_rows_fwd<N_>(fa, fb, nz, oa, ob, tw, s)))
}
cudaError_t rows_inv_any(int nx, const cx<float>* ia, int nz, float scale, float* fa, const cx<float>* tw, cudaStream_t s) {
    ZK_STATIC_SWITCH(nx, (s_rows_inv<N_>(ia, nz, scale, fa, tw, s)))
}
template <bool INV>
cudaError_t cols_any(int nz, cx<float>* f0, cx<float>* f1, int hx, const cx<float>* tw, cudaStream_t s) {
    ZK_STATIC_SWITCH(nz, (s_cols<N_, INV>(f0, f1, hx, tw, s)))
}

bool pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }

cudaError_t dno_static(unsigned char* base, const Layout& L, const float* eta, const float* psi, float* v,
                       int nx, int nz, double Lx, double Lz, double h, double g, int M, double eps, int taper,
                       cudaStream_t s) {
    const int npx = 3 * nx / 2, npz = 3 * nz / 2, hx = nx / 2;
    auto C = [&](size_t off) { return reinterpret_cast<cx<float>*>(base + off); };
    cx<float>* twx = C(L.tw_x);
    cx<float>* twz = C(L.tw_z);
    cx<float>* twpx = C(L.tw_px);
    cx<float>* twpz = C(L.tw_pz);
    cx<float>* ye = C(L.y_eta);
    cx<float>* yp = C(L.y_psi);
    cx<float>* ke = C(L.ko_eta);
    cx<float>* kp = C(L.ko_psi);
    cx<float>* col = C(L.col);
    float* acc = reinterpret_cast<float*>(base + L.acc);
    const long long fstride = (long long)npz * hx;
    cudaError_t e;
    // the previous call's contents are not trusted: clear the spectra this call accumulates into
    const size_t comp = (size_t)nz * hx * sizeof(cx<float>);
    if ((e = cudaMemsetAsync(ye, 0, comp, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(yp, 0, comp, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ke, 0, comp, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(kp, 0, comp, s)) != cudaSuccess) return e;
    const int ns[4] = {nx, nz, npx, npz};
    cx<float>* tws[4] = {twx, twz, twpx, twpz};
    for (int i = 0; i < 4; ++i) {
        if (i < 2) {
            static_twiddle_kernel<<<(ns[i] + 127) / 128, 128, 0, s>>>(tws[i], ns[i]);
        } else {
            const PlanDesc d = plan_desc_of(ns[i]);
            const int ne = plan_table_size(d);
            static_plan_twiddle_kernel<<<(ne + 127) / 128, 128, 0, s>>>(tws[i], d, ne);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // physical -> compact spectra
    if ((e = rows_fwd_any(nx, eta, psi, nz, ye, yp, twx, s)) != cudaSuccess) return e;
    if ((e = cols_any<false>(nz, ye, yp, hx, twz, s)) != cudaSuccess) return e;

    const SFields F{M};
    ColArgs<float> cb;
    std::memset(&cb, 0, sizeof(cb));
    cb.hx = hx; cb.nz_grid = nz; cb.nx_grid = nx;
    cb.kx0 = (float)(2.0 * M_PI / Lx); cb.kz0 = (float)(2.0 * M_PI / Lz);
    cb.h = (float)h; cb.g = (float)g;
    cb.kc = (float)(2.0 / 3.0 * M_PI / std::max(Lx / nx, Lz / nz));
    cb.taper = taper;
    cb.fscale = (float)((double)nx * nz / ((double)npx * npz));
    cb.iscale = (float)(1.0 / ((double)nx * nz));
    cb.colbase = col; cb.fstride = fstride;
    RowArgs<float> rb;
    std::memset(&rb, 0, sizeof(rb));
    rb.colbase = col; rb.fstride = fstride; rb.M = M; rb.eps = (float)eps;
    double p = 1.0;
    for (int j = 0; j < kMaxOrder + 3; ++j) { rb.epsp[j] = (float)p; p *= eps; }
    rb.kx0 = (float)(2.0 * M_PI / Lx);
    rb.acc = acc;
    rb.s_eta = rb.s_etax = rb.s_etaz = rb.s_psix = rb.s_psiz = rb.s_g0psi = rb.s_F0 = -1;
    for (int l = 0; l < kMaxLines; ++l) { rb.fa[l] = -1; rb.fb[l] = -1; }
    struct Slots {
        RowArgs<float>* a; int n = 0;
        int add(int f, bool dx) {
            const int l = n >> 1;
            if (n & 1) { a->fb[l] = f; if (dx) a->dxb |= 1u << l; } else { a->fa[l] = f; if (dx) a->dxa |= 1u << l; }
            return n++;
        }
        void finish() { a->nlines = (n + 1) >> 1; }
    };
    {   // round 0
        ColArgs<float> a = cb;
        a.kind = COL_FROM_STATE; a.st_eta = ye; a.st_psi = yp;
        int o = 0;
        auto out = [&](int f, int src, int sym, int aa) { a.out_f[o] = f; a.out_src[o] = src; a.out_sym[o] = sym; a.out_a[o] = aa; ++o; };
        out(0, 0, SYM_ID, 0); out(1, 0, SYM_DZ, 0); out(2, 1, SYM_ID, 0); out(3, 1, SYM_DZ, 0);
        for (int q = 1; q <= M; ++q) out(F.z(0, q), 1, SYM_ZA, q);
        a.nout = o;
        if ((e = s_col_any(npz, a, twpz, s)) != cudaSuccess) return e;
    }
    for (int r = 1; r <= M - 1; ++r) {
        RowArgs<float> ra = rb;
        ra.kind = 0; ra.r = r;
        Slots sl{&ra};
        ra.s_eta = sl.add(0, false);
        if (r >= 2 && r - 1 <= M - 3) { ra.s_etax = sl.add(0, true); ra.s_etaz = sl.add(1, false); }
        ra.s_F0 = sl.n;
        for (int j = 0; j < r; ++j) sl.add(F.z(j, r - j), false);
        sl.finish();
        ra.out0 = col + (long long)F.phiout() * fstride;
        if ((e = s_row_any(npx, ra, twpx, npz, s)) != cudaSuccess) return e;
        ColArgs<float> a = cb;
        a.kind = COL_PHI; a.pin = col + (long long)F.phiout() * fstride;
        int o = 0;
        for (int q = 1; q <= M - r; ++q) { a.out_f[o] = F.z(r, q); a.out_src[o] = 0; a.out_sym[o] = SYM_ZA; a.out_a[o] = q; ++o; }
        a.nout = o;
        if ((e = s_col_any(npz, a, twpz, s)) != cudaSuccess) return e;
    }
    {   // final round
        RowArgs<float> ra = rb;
        ra.kind = 1; ra.r = M;
        Slots sl{&ra};
        if (M >= 2) ra.s_eta = sl.add(0, false);
        ra.s_etax = sl.add(0, true); ra.s_etaz = sl.add(1, false);
        ra.s_psix = sl.add(2, true); ra.s_psiz = sl.add(3, false);
        ra.s_g0psi = sl.add(F.z(0, 1), false);
        if (M >= 2) { ra.s_F0 = sl.n; for (int j = 0; j < M; ++j) sl.add(F.z(j, M - j), false); }
        sl.finish();
        ra.out0 = col + (long long)F.gnl() * fstride;
        ra.out1 = col + (long long)F.npsi() * fstride;
        if ((e = s_row_any(npx, ra, twpx, npz, s)) != cudaSuccess) return e;
        ColArgs<float> a = cb;
        a.kind = COL_FINAL; a.mode = FIN_RHS;
        a.gin = col + (long long)F.gnl() * fstride;
        a.nin = col + (long long)F.npsi() * fstride;
        a.s_eta = ye; a.s_psi = yp; a.ko_eta = ke; a.ko_psi = kp;
        if ((e = s_col_any(npz, a, twpz, s)) != cudaSuccess) return e;
    }
    // compact G psi -> physical output
    if ((e = cols_any<true>(nz, ke, nullptr, hx, twz, s)) != cudaSuccess) return e;
    return rows_inv_any(nx, ke, nz, (float)(1.0 / ((double)nx * nz)), v, twx, s);
}

}  // namespace

extern "C" zk_status zk_dno_static(const float* eta, const float* psi, float* v, int nx, int nz, double Lx,
                                   double Lz, double h, double g, int M, double eps, int taper, void* stream) {
    if (!eta || !psi || !v) return ZK_EINVAL;
    if (!pow2_in(nx, 16, 256) || !pow2_in(nz, 16, 256)) return ZK_EINVAL;
    if (M < 1 || M > ZK_MAX_ORDER) return ZK_EINVAL;
    if (!(Lx > 0) || !(Lz > 0) || !(h > 0) || !(g > 0) || !(eps >= 0.0 && eps <= 1.0)) return ZK_EINVAL;
    if (taper != 0 && taper != 1) return ZK_EINVAL;
    const Layout L = layout(nx, nz, M);
    if (L.total > (size_t)ZK_STATIC_SCRATCH_BYTES) return ZK_EINVAL;
    void* base = nullptr;
    const zk_status st = scratch_address(&base);
    if (st != ZK_OK) return st;
    const cudaError_t e = dno_static(static_cast<unsigned char*>(base), L, eta, psi, v, nx, nz, Lx, Lz, h, g, M,
                                     eps, taper, (cudaStream_t)stream);
    return e == cudaSuccess ? ZK_OK : ZK_ECUDA;
}
