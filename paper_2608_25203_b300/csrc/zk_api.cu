// zk_api.cu - the C ABI of include/zk.h: context, device buffers, launch order.
//
// One right-hand side at order M is 2M+1 launches (Sec. 3.2 recursion, one
// de-aliased grid per evaluation, Sec. 6.1):
//   col(kind 0) -> [row(r) -> col(kind 1, r)] for r = 1..M-1 -> row(final) -> col(final)
// An RK4 step is four of them; the final column kernel of each stage does the
// stage combination, and the last one also applies the state filter (Eq. 17).
// On 1536-point and longer columns the final column kernel ends with its
// transforms and a separate update launch (fin_epilogue_kernel) does the rest.
// zk_step captures the launches of one step into a CUDA graph (re-captured
// when dt or the options change) and replays it n times on the context's
// stream.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <algorithm>
#include <unordered_map>
#include <vector>

#include "../../include/zk.h"
#include "zk_kernels2.cuh"
#include "zk_launch.h"
#include "zk_net_internal.h"

using namespace zk;

namespace {

constexpr int kIoElem = 8;  // bytes per staging element (fits f32 and f64)

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

}  // namespace

struct zk_ctx {
    int nx = 0, nz = 0, npx = 0, npz = 0, hx = 0, M = 0, prec = ZK_F32;
    double Lx = 0, Lz = 0, h = 0, g = 0;
    zk_options opt{};
    int device = 0;
    bool has_state = false;
    size_t csz = 0;  // bytes per complex element
    void *tw_x = nullptr, *tw_z = nullptr, *tw_px = nullptr, *tw_pz = nullptr;
    void* tw_pv[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   // padded plan tables [variant][x, z]
    // half-length plan tables of the padded rows [variant] (nullptr where the plan of npx has
    // no half-length form) and w_npx^k, k < npx/2: the real forward row transform at half length
    void* tw_hv[2] = {nullptr, nullptr};
    void* tw_rx = nullptr;
    // tiles sharing this grid and order (a batch group; 1 for a plain context):
    // buffers are [tile][...] with these element strides, depth per tile
    int nb = 1;
    long long tcol = 0, tst = 0, tacc = 0;
    void* hb = nullptr;                    // device [nb] depths in the compute type (nb > 1)
    std::vector<double> hv;                // host copy of the depths
    // launch shape (set by the batch autotuner): plan variant, columns-per-block
    // choice (0 / 1 / 2 = half / default / double), row blocks per SM (0 = all resident)
    int plan_v = 0, col_ci = 1, row_occ = 0;
    int dft_split = 0;                     // ZK_DFT_*: innermost radix-8 stage on the tensor cores
    int m_run = 0;                         // order of the right-hand side being enqueued (<= M)
    bool series64 = false;                 // FP32 context: series sums and accumulator in FP64
    bool pad3 = false;                     // padded grid 3N (exact series products) instead of 3N/2
    // asynchronous host I/O: copies on their own stream through two staging slots per direction
    cudaStream_t io = nullptr, io_out = nullptr;   // uploads, downloads (separate, so that they overlap)
    cudaEvent_t ev_in[2] = {}, ev_in_used[2] = {}, ev_out[2] = {}, ev_out_done[2] = {};
    bool in_used_rec[2] = {false, false}, out_done_rec[2] = {false, false};
    void* astage_in[2] = {nullptr, nullptr};
    void* astage_out[2] = {nullptr, nullptr};
    int in_slot = 0, out_slot = 0;
    // learned closure (FP32): order-base_M right-hand side plus the network's residual
    zk_net* net = nullptr;
    bool closure_on = false;
    bool closure_once = false;   // evaluate the network at the first RK stage only, reuse it after
    int base_M = 2;
    ClosureScales sc{};
    int check_every = 0;
    double check_tol = 0.2;
    int nchecks = 0;
    long long nsteps = 0;                  // steps taken since the closure was set
    long long fallback_step = -1;
    double last_err = -1.0;
    void* cspec = nullptr;                 // 6 compact spectra (features, then the residual)
    void* feat = nullptr;                  // [6][nz][nx] FP32 features
    void* rbuf = nullptr;                  // [2][nz][nx] FP32 network output
    void* chk = nullptr;                   // 2 compact spectra: the high-order right-hand side
    double* cpart = nullptr;               // check partial sums
    // adaptive order: every adapt_every steps pick the smallest order in
    // [adapt_min, M] whose right-hand side is within adapt_tol of order M's
    int adapt_every = 0, adapt_min = 1, adapt_checks = 0;
    double adapt_tol = 0.0;
    double adapt_err[ZK_MAX_ORDER + 1] = {};
    void *y_eta = nullptr, *y_psi = nullptr, *ys_eta = nullptr, *ys_psi = nullptr;
    void *ka_eta = nullptr, *ka_psi = nullptr, *ko_eta = nullptr, *ko_psi = nullptr;
    void *h_eta = nullptr, *h_psi = nullptr;   // IF-AB2 forcing history
    bool ab_valid = false;                     // history holds F_{n-1} taken at ab_dt
    double ab_dt = 0.0;
    void *col = nullptr;
    int nfields = 0;
    long long fstride = 0;
    void *acc = nullptr;
    void *sfc = nullptr;       // surface planes eta, dx eta, dz eta: [3][npz][npx] real per tile
    void *fsc = nullptr;       // final pass, split: transformed nonlinear parts Fe, Fp (2 compact per tile)
    void *stage = nullptr;
    void *tank = nullptr;      // two (nx/2) x (nz/2) FP64-sized arrays for tank I/O
    double *partial = nullptr;
    int npartial = 0;
    double *esum = nullptr;
    size_t bytes = 0;
    std::vector<void*> allocs;
    // graph of one step
    cudaStream_t cap = nullptr;
    cudaGraphExec_t gexec = nullptr;      // RK4 step, or IF-AB2 step with history
    cudaGraphExec_t gexec_boot = nullptr; // IF-AB2 bootstrap step (IF-Euler)
    bool gvalid = false;
    double gdt = 0.0;
    int launches_per_step = 0;
    int fin_blocks = 0;      // blocks of the last final column kernel (energy partials)
    // per-launch profiling (zk_profile_step): events recorded before each launch
    std::vector<cudaEvent_t>* prof_ev = nullptr;
    std::vector<int> slot_kind;
    std::vector<double> slot_bytes;
};

namespace {

cudaStream_t user_stream(const zk_ctx* c) { return (cudaStream_t)c->opt.stream; }
// Plan variant of the padded transforms: the split-precision DFT-GEMM plans
// (SPLIT_BF16 / SPLIT_FP16) when selected, else the tuned FP32 plan.
int plan_of(const zk_ctx* c) {
    return c->dft_split == ZK_DFT_BF16X3 ? SPLIT_BF16 : c->dft_split == ZK_DFT_FP16X3 ? SPLIT_FP16 : c->plan_v;
}
void drop_graph(zk_ctx* c);

zk_status cu(cudaError_t e) { return e == cudaSuccess ? ZK_OK : ZK_ECUDA; }

// Column-space field indices.
struct Fields {
    int M;
    int eta() const { return 0; }
    int dzeta() const { return 1; }
    int psi() const { return 2; }
    int dzpsi() const { return 3; }
    int base(int j) const {  // first dz^a Phi(j) field, j >= 1
        int b = 4 + M;
        for (int r = 1; r < j; ++r) b += M - r;
        return b;
    }
    int z(int j, int a) const { return j == 0 ? 3 + a : base(j) + a - 1; }
    int phiout() const { return base(M); }
    int gnl() const { return phiout() + 1; }
    int npsi() const { return phiout() + 2; }
    int count() const { return phiout() + 3; }
};

template <typename T>
void make_twiddles(int n, std::vector<cx<T>>& out) {
    out.resize(n);
    for (int t = 0; t < n; ++t) {
        const double ang = -2.0 * M_PI * (double)t / (double)n;
        out[t] = mk<T>((T)std::cos(ang), (T)std::sin(ang));
    }
}

template <typename T, typename TIN, int NX>
cudaError_t launch_rows_fwd_t(const void* fa, const void* fb, int nz, cx<T>* oa, cx<T>* ob, const cx<T>* tw, cudaStream_t s) {
    constexpr int TL = Plan<NX>::TL;
    const int threads = TL >= 128 ? TL : 128;
    const int rows = threads / TL;
    const size_t smem = (size_t)rows * line_stride(NX) * sizeof(cx<T>);
    cudaError_t e = ensure_smem((const void*)rows_fwd_kernel<T, TIN, NX>, smem);
    if (e != cudaSuccess) return e;
    rows_fwd_kernel<T, TIN, NX><<<(nz + rows - 1) / rows, threads, smem, s>>>((const TIN*)fa, (const TIN*)fb, nz, oa, ob, tw);
    return cudaGetLastError();
}
template <typename T, typename TOUT, int NX>
cudaError_t launch_rows_inv_t(const cx<T>* ia, const cx<T>* ib, int nz, T scale, void* fa, void* fb, const cx<T>* tw, cudaStream_t s) {
    constexpr int TL = Plan<NX>::TL;
    const int threads = TL >= 128 ? TL : 128;
    const int rows = threads / TL;
    const size_t smem = (size_t)rows * line_stride(NX) * sizeof(cx<T>);
    cudaError_t e = ensure_smem((const void*)rows_inv_kernel<T, TOUT, NX>, smem);
    if (e != cudaSuccess) return e;
    rows_inv_kernel<T, TOUT, NX><<<(nz + rows - 1) / rows, threads, smem, s>>>(ia, ib, nz, scale, (TOUT*)fa, (TOUT*)fb, tw);
    return cudaGetLastError();
}
template <typename T, int NZ, bool INV>
cudaError_t launch_cols_t(cx<T>* f0, cx<T>* f1, int hx, const cx<T>* tw, cudaStream_t s) {
    constexpr int CB = cols_cb<NZ>(), threads = CB * Plan<NZ>::TL;
    constexpr size_t smem = cols_smem_bytes<T, NZ>();
    cudaError_t e = ensure_smem((const void*)cols_kernel<T, NZ, INV>, smem);
    if (e != cudaSuccess) return e;
    cols_kernel<T, NZ, INV><<<(hx + CB - 1) / CB, threads, smem, s>>>(f0, f1, hx, tw);
    return cudaGetLastError();
}

template <typename T, typename TIN, int NX>
cudaError_t launch_relax_rows_t(cx<T>* f, const void* sigma, const void* target, int nz, T dt, T scale,
                                const cx<T>* tw, cudaStream_t s) {
    constexpr int TL = Plan<NX>::TL;
    const int threads = TL >= 128 ? TL : 128;
    const int rows = threads / TL;
    const size_t smem = (size_t)rows * line_stride(NX) * sizeof(cx<T>);
    cudaError_t e = ensure_smem((const void*)relax_rows_kernel<T, TIN, NX>, smem);
    if (e != cudaSuccess) return e;
    relax_rows_kernel<T, TIN, NX><<<(nz + rows - 1) / rows, threads, smem, s>>>(
        f, (const TIN*)sigma, (const TIN*)target, nz, dt, scale, tw);
    return cudaGetLastError();
}

#define ZK_SWITCH_N(n, CALL)                                     \
    switch (n) {                                                 \
    case 16: { constexpr int N_ = 16; return CALL; }             \
    case 32: { constexpr int N_ = 32; return CALL; }             \
    case 64: { constexpr int N_ = 64; return CALL; }             \
    case 128: { constexpr int N_ = 128; return CALL; }           \
    case 256: { constexpr int N_ = 256; return CALL; }           \
    case 512: { constexpr int N_ = 512; return CALL; }           \
    case 1024: { constexpr int N_ = 1024; return CALL; }         \
    case 2048: { constexpr int N_ = 2048; return CALL; }         \
    default: return cudaErrorInvalidValue;                       \
    }

template <typename T, typename TIN>
cudaError_t launch_rows_fwd(int nx, const void* fa, const void* fb, int nz, cx<T>* oa, cx<T>* ob, const cx<T>* tw, cudaStream_t s) {
    ZK_SWITCH_N(nx, (launch_rows_fwd_t<T, TIN, N_>(fa, fb, nz, oa, ob, tw, s)))
}
template <typename T, typename TOUT>
cudaError_t launch_rows_inv(int nx, const cx<T>* ia, const cx<T>* ib, int nz, T scale, void* fa, void* fb, const cx<T>* tw, cudaStream_t s) {
    ZK_SWITCH_N(nx, (launch_rows_inv_t<T, TOUT, N_>(ia, ib, nz, scale, fa, fb, tw, s)))
}
template <typename T, typename TIN>
cudaError_t launch_relax_rows(int nx, cx<T>* f, const void* sigma, const void* target, int nz, T dt, T scale,
                              const cx<T>* tw, cudaStream_t s) {
    ZK_SWITCH_N(nx, (launch_relax_rows_t<T, TIN, N_>(f, sigma, target, nz, dt, scale, tw, s)))
}
template <typename T, bool INV>
cudaError_t launch_cols(int nz, cx<T>* f0, cx<T>* f1, int hx, const cx<T>* tw, cudaStream_t s) {
    ZK_SWITCH_N(nz, (launch_cols_t<T, N_, INV>(f0, f1, hx, tw, s)))
}

// ---------------------------------------------------------------------------
// The right-hand-side pipeline.
// ---------------------------------------------------------------------------
template <typename T>
struct Pipe {
    static cx<T>* C(void* p) { return reinterpret_cast<cx<T>*>(p); }

    static ColArgs<T> col_base(const zk_ctx* c) {
        ColArgs<T> a;
        std::memset(&a, 0, sizeof(a));
        a.hx = c->hx;
        a.nz_grid = c->nz;
        a.nx_grid = c->nx;
        a.kx0 = (T)(2.0 * M_PI / c->Lx);
        a.kz0 = (T)(2.0 * M_PI / c->Lz);
        a.h = (T)c->h;
        a.g = (T)c->g;
        const double dmax = std::max(c->Lx / c->nx, c->Lz / c->nz);
        a.kc = (T)(2.0 / 3.0 * M_PI / dmax);
        a.taper = c->opt.taper;
        a.fscale = (T)((double)c->nx * c->nz / ((double)c->npx * c->npz));
        a.iscale = (T)(1.0 / ((double)c->nx * c->nz));
        a.colbase = C(c->col);
        a.fstride = c->fstride;
        a.filter = c->opt.filter;
        a.tcol = c->tcol;
        a.tst = c->tst;
        a.hb = reinterpret_cast<const T*>(c->hb);
        a.nb = c->nb;
        a.pad3 = c->pad3 ? 1 : 0;
        return a;
    }

    static RowArgs<T> row_base(const zk_ctx* c) {
        RowArgs<T> a;
        std::memset(&a, 0, sizeof(a));
        a.colbase = C(c->col);
        a.fstride = c->fstride;
        a.M = c->m_run > 0 ? c->m_run : c->M;
        a.eps = (T)c->opt.eps;
        double p = 1.0;
        for (int j = 0; j < kMaxOrder + 3; ++j) { a.epsp[j] = (T)p; p *= c->opt.eps; }
        a.kx0 = (T)(2.0 * M_PI / c->Lx);
        a.acc = reinterpret_cast<T*>(c->acc);
        a.s_eta = a.s_etax = a.s_etaz = a.s_psix = a.s_psiz = a.s_g0psi = a.s_F0 = -1;
        for (int l = 0; l < kMaxLines; ++l) { a.fa[l] = -1; a.fb[l] = -1; }
        a.tcol = c->tcol;
        a.tacc = c->tacc;
        a.nb = c->nb;
        a.occ = c->row_occ;
        a.acc64 = (sizeof(T) == 4 && c->series64) ? 1 : 0;
        a.pad3 = c->pad3 ? 1 : 0;
        a.sfc = reinterpret_cast<T*>(c->sfc);
        a.tsfc = 3 * c->tacc;
        a.sfc_mode = 0;
        // half-length real forward transform: plans 0 / 1 only (the split-precision plans keep
        // the full-length transform); the kernel falls back where its block shape does not fit
        const int pv = plan_of(c);
        a.twh = (pv == 0 || pv == 1) && c->tw_rx ? reinterpret_cast<const cx<T>*>(c->tw_hv[pv]) : nullptr;
        a.twr = a.twh ? reinterpret_cast<const cx<T>*>(c->tw_rx) : nullptr;
        return a;
    }

    // slot list helper: appends a real field (field index, dx flag) and returns its slot
    struct Slots {
        RowArgs<T>* a;
        int n = 0;
        int add(int f, bool dx) {
            const int l = n >> 1;
            if (n & 1) { a->fb[l] = f; if (dx) a->dxb |= 1u << l; }
            else { a->fa[l] = f; if (dx) a->dxa |= 1u << l; }
            return n++;
        }
        void finish() { a->nlines = (n + 1) >> 1; }
    };

    // Enqueue one right-hand side at state (se, sp); the final column kernel
    // runs `mode` with the given epilogue arguments already in `fin`.
    // Record the profiling event of the next launch, with its class and its
    // algorithmic bytes (each input field read once, each output written once).
    static void note(zk_ctx* c, cudaStream_t s, int kind, double bytes) {
        if (!c->prof_ev) return;
        cudaEvent_t ev;
        cudaEventCreate(&ev);
        cudaEventRecord(ev, s);
        c->prof_ev->push_back(ev);
        c->slot_kind.push_back(kind);
        c->slot_bytes.push_back(bytes);
    }

    static cudaError_t rhs(zk_ctx* c, const cx<T>* se, const cx<T>* sp, ColArgs<T> fin, cudaStream_t s, int* nlaunch) {
        const int M = c->m_run > 0 ? c->m_run : c->M;
        const Fields F{M};
        const double U = (double)c->fstride * sizeof(cx<T>);                 // one column-space field
        const double Cc = (double)c->nz * c->hx * sizeof(cx<T>);             // one compact spectrum
        const double Pp = (double)c->npz * c->npx * sizeof(T);               // the padded accumulator
        const cx<T>* twx = reinterpret_cast<const cx<T>*>(c->tw_px);
        const cx<T>* twz = reinterpret_cast<const cx<T>*>(c->tw_pz);
        cudaError_t e;
        int nl = 0;
        // round 0: state -> column space
        {
            ColArgs<T> a = col_base(c);
            a.kind = COL_FROM_STATE;
            a.st_eta = se;
            a.st_psi = sp;
            int o = 0;
            auto out = [&](int f, int src, int sym, int aa) {
                a.out_f[o] = f; a.out_src[o] = src; a.out_sym[o] = sym; a.out_a[o] = aa; ++o;
            };
            out(F.eta(), 0, SYM_ID, 0);
            out(F.dzeta(), 0, SYM_DZ, 0);
            out(F.psi(), 1, SYM_ID, 0);
            out(F.dzpsi(), 1, SYM_DZ, 0);
            for (int q = 1; q <= M; ++q) out(F.z(0, q), 1, SYM_ZA, q);
            a.nout = o;
            note(c, s, ZK_K_COL_STATE, 2 * Cc + o * U);
            if ((e = launch_col<T>(c->npz, plan_of(c), c->col_ci, a, twz, s)) != cudaSuccess) return e;
            ++nl;
        }
        // Surface planes (every order M >= 2): round 1 transforms eta, dx eta and dz eta once
        // and writes them; the later rounds and the final round read them.
        const bool sfc = c->sfc != nullptr && M >= 2;
        const double Ps = (double)c->npz * c->npx * sizeof(T);                // one surface plane
        for (int r = 1; r <= M - 1; ++r) {
            RowArgs<T> ra = row_base(c);
            ra.kind = 0;
            ra.r = r;
            Slots sl{&ra};
            const bool g2 = r >= 2 && r - 1 <= M - 3;   // the round uses the slopes of eta
            if (sfc && r == 1) {
                ra.sfc_mode = 1;
                ra.s_eta = sl.add(F.eta(), false);
                ra.s_etax = sl.add(F.eta(), true);
                ra.s_etaz = sl.add(F.dzeta(), false);
            } else if (sfc) {
                ra.sfc_mode = 2;
            } else {
                ra.s_eta = sl.add(F.eta(), false);
                if (g2) {
                    ra.s_etax = sl.add(F.eta(), true);
                    ra.s_etaz = sl.add(F.dzeta(), false);
                }
            }
            ra.s_F0 = sl.n;
            for (int j = 0; j < r; ++j) sl.add(F.z(j, r - j), false);
            sl.finish();
            ra.out0 = C(c->col) + (long long)F.phiout() * c->fstride;
            {
                double rd, wr = U + (r >= 2 ? Pp : 0.0);
                if (!sfc) rd = (1 + (g2 ? 1 : 0) + r) * U;
                else if (r == 1) { rd = 2 * U + r * U; wr += 3 * Ps; }
                else rd = r * U + (g2 ? 3 : 1) * Ps;
                if (r >= 3) rd += Pp;
                note(c, s, ZK_K_ROW_ROUND, rd + wr);
            }
            if ((e = launch_row<T>(c->npx, plan_of(c), ra, twx, c->npz, s)) != cudaSuccess) return e;
            ++nl;
            ColArgs<T> a = col_base(c);
            a.kind = COL_PHI;
            a.pin = C(c->col) + (long long)F.phiout() * c->fstride;
            int o = 0;
            for (int q = 1; q <= M - r; ++q) {
                a.out_f[o] = F.z(r, q); a.out_src[o] = 0; a.out_sym[o] = SYM_ZA; a.out_a[o] = q; ++o;
            }
            a.nout = o;
            note(c, s, ZK_K_COL_PHI, (1 + o) * U);
            if ((e = launch_col<T>(c->npz, plan_of(c), c->col_ci, a, twz, s)) != cudaSuccess) return e;
            ++nl;
        }
        {
            RowArgs<T> ra = row_base(c);
            ra.kind = 1;
            ra.r = M;
            Slots sl{&ra};
            if (sfc) {
                ra.sfc_mode = 2;
            } else {
                if (M >= 2) ra.s_eta = sl.add(F.eta(), false);
                ra.s_etax = sl.add(F.eta(), true);
                ra.s_etaz = sl.add(F.dzeta(), false);
            }
            ra.s_psix = sl.add(F.psi(), true);
            ra.s_psiz = sl.add(F.dzpsi(), false);
            ra.s_g0psi = sl.add(F.z(0, 1), false);
            if (M >= 2) {
                ra.s_F0 = sl.n;
                for (int j = 0; j < M; ++j) sl.add(F.z(j, M - j), false);
            }
            sl.finish();
            ra.out0 = C(c->col) + (long long)F.gnl() * c->fstride;
            ra.out1 = C(c->col) + (long long)F.npsi() * c->fstride;
            note(c, s, ZK_K_ROW_FINAL,
                 (sfc ? 3 * U + 3 * Ps : 5 * U) + ((M >= 2 ? M : 0) + 2) * U + (M >= 3 ? Pp : 0.0));
            if ((e = launch_row<T>(c->npx, plan_of(c), ra, twx, c->npz, s)) != cudaSuccess) return e;
            ++nl;
        }
        {
            fin.kind = COL_FINAL;
            fin.gin = C(c->col) + (long long)F.gnl() * c->fstride;
            fin.nin = C(c->col) + (long long)F.npsi() * c->fstride;
            fin.s_eta = se;
            fin.s_psi = sp;
            // Long columns: the update runs as its own launch over the compact spectra (the column
            // kernel's one block per SM would wait on the stage state's global loads).
            const bool split = c->fsc != nullptr && c->npz >= 1536 && fin.mode != FIN_ENERGY;
            double b_epi = 0.0;
            {
                // 2 products in, the stage state, then the epilogue's own traffic
                double b = 2 * U + 2 * Cc;
                switch (fin.mode) {
                case FIN_RHS: b += 2 * Cc; break;
                case FIN_RK1: b += 4 * Cc; break;                 // ka, ys written (state is y)
                case FIN_RK2: case FIN_RK3: b += 8 * Cc; break;   // y, ka read; ka, ys written
                case FIN_RK4: b += 6 * Cc; break;                 // y, ka read; y written
                case FIN_IRK1: b += 6 * Cc; break;                // y read; ka, ys written
                case FIN_IRK2: case FIN_IRK3: b += 8 * Cc; break; // y, ka read; ka, ys written
                case FIN_IRK4: b += 6 * Cc; break;                // y, ka read; y written
                default: break;
                }
                if (split) {
                    // transforms: products in, Fe and Fp out; update: Fe, Fp, the state and the rest
                    b_epi = b - 2 * U + 2 * Cc;
                    b = 2 * U + 2 * Cc;
                }
                note(c, s, ZK_K_COL_FINAL, b);
            }
            if (split) {
                fin.split = 1;
                fin.fe = reinterpret_cast<cx<T>*>(c->fsc);
                fin.fp = fin.fe + (long long)c->nz * c->hx * c->nb;   // [tile][nz][hx] each
            }
            if ((e = launch_col<T>(c->npz, plan_of(c), c->col_ci, fin, twz, s, &c->fin_blocks)) != cudaSuccess) return e;
            ++nl;
            if (split) {
                note(c, s, ZK_K_COL_FINAL, b_epi);
                const long long n = (long long)c->nz * c->hx;
                const int blocks = (int)std::min<long long>((n + 255) / 256, 148LL * 16);
                fin_epilogue_kernel<T><<<dim3(blocks, std::max(1, c->nb)), 256, 0, s>>>(fin);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
                ++nl;
            }
        }
        if (nlaunch) *nlaunch += nl;
        return cudaSuccess;
    }

    static cudaError_t rk4_step(zk_ctx* c, double dt, cudaStream_t s, int* nlaunch) {
        for (int st = 1; st <= 4; ++st) {
            ColArgs<T> fin = col_base(c);
            fin.mode = st;
            fin.dt = (T)dt;
            fin.y_eta = C(c->y_eta); fin.y_psi = C(c->y_psi);
            fin.ys_eta = C(c->ys_eta); fin.ys_psi = C(c->ys_psi);
            fin.ka_eta = C(c->ka_eta); fin.ka_psi = C(c->ka_psi);
            const cx<T>* se = st == 1 ? C(c->y_eta) : C(c->ys_eta);
            const cx<T>* sp = st == 1 ? C(c->y_psi) : C(c->ys_psi);
            cudaError_t e = rhs(c, se, sp, fin, s, nlaunch);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }

    // ---- learned closure (FP32 contexts) -------------------------------------
    // Residual spectra R_hat (unnormalised, both components) into cspec[0..1]
    // from the state (se, sp) and the low-order right-hand side held in ko.
    static cudaError_t closure_residual(zk_ctx* c, const cx<T>* se, const cx<T>* sp, cudaStream_t s, int* nl) {
        const long long n = (long long)c->nz * c->hx;
        cx<T>* cs = C(c->cspec);
        closure_prep_kernel<T><<<4 * 148, 256, 0, s>>>(se, sp, C(c->ko_eta), C(c->ko_psi), cs, c->nz, c->hx,
                                                       (T)(2.0 * M_PI / c->Lx), (T)(2.0 * M_PI / c->Lz), (T)c->h,
                                                       (T)c->g, c->sc);
        cudaError_t e = cudaGetLastError();
        float* f = reinterpret_cast<float*>(c->feat);
        const size_t plane = (size_t)c->nx * c->nz;
        for (int k = 0; k < 3 && e == cudaSuccess; ++k)
            e = to_physical(c, cs + 2 * k * n, cs + (2 * k + 1) * n, f + 2 * k * plane, f + (2 * k + 1) * plane, ZK_F32, s);
        const float* y = nullptr;
        if (e == cudaSuccess) e = zk_net_infer(c->net, f, &y, 1, c->nz, c->nx, s);
        const cx<T>* twx = reinterpret_cast<const cx<T>*>(c->tw_x);
        const cx<T>* twz = reinterpret_cast<const cx<T>*>(c->tw_z);
        if (e == cudaSuccess) e = launch_rows_fwd<T, float>(c->nx, y, y + plane, c->nz, cs, cs + n, twx, s);
        if (e == cudaSuccess) e = launch_cols<T, false>(c->nz, cs, cs + n, c->hx, twz, s);
        if (nl) *nl += 1 + 6 + 4 + 2;
        return e;
    }

    // One closure right-hand side at (se, sp): order-base_M right-hand side,
    // the residual, and the combination/epilogue of `fin` (mode set by the caller).
    // With reuse, the residual spectrum of the previous evaluation (held in cspec) is applied
    // again instead of evaluating the network at this state.
    static cudaError_t closure_stage(zk_ctx* c, const cx<T>* se, const cx<T>* sp, ColArgs<T> fin, cudaStream_t s, int* nl,
                                     bool reuse = false) {
        ColArgs<T> r = col_base(c);
        r.mode = FIN_RHS;
        r.ko_eta = C(c->ko_eta);
        r.ko_psi = C(c->ko_psi);
        const int save = c->m_run;
        c->m_run = c->base_M;
        cudaError_t e = rhs(c, se, sp, r, s, nl);
        c->m_run = save;
        if (e == cudaSuccess && !reuse) e = closure_residual(c, se, sp, s, nl);
        if (e == cudaSuccess) {
            const long long n = (long long)c->nz * c->hx;
            fin.ko_eta = C(c->ko_eta);
            fin.ko_psi = C(c->ko_psi);
            closure_combine_kernel<T><<<4 * 148, 256, 0, s>>>(fin, C(c->cspec), C(c->cspec) + n, c->sc);
            e = cudaGetLastError();
            if (nl) ++*nl;
        }
        return e;
    }

    static cudaError_t closure_rk4_step(zk_ctx* c, double dt, cudaStream_t s, int* nlaunch) {
        for (int st = 1; st <= 4; ++st) {
            ColArgs<T> fin = col_base(c);
            fin.mode = st;
            fin.dt = (T)dt;
            fin.y_eta = C(c->y_eta); fin.y_psi = C(c->y_psi);
            fin.ys_eta = C(c->ys_eta); fin.ys_psi = C(c->ys_psi);
            fin.ka_eta = C(c->ka_eta); fin.ka_psi = C(c->ka_psi);
            const cx<T>* se = st == 1 ? C(c->y_eta) : C(c->ys_eta);
            const cx<T>* sp = st == 1 ? C(c->y_psi) : C(c->ys_psi);
            cudaError_t e = closure_stage(c, se, sp, fin, s, nlaunch, c->closure_once && st > 1);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }

    // Fallback check at the current state: relative L2 error of the predicted
    // residual against f_M - f_base (both components); past check_tol the
    // closure is switched off and the context steps at order M from then on.
    static zk_status closure_check(zk_ctx* c, cudaStream_t s) {
        const long long n = (long long)c->nz * c->hx;
        const size_t compact = (size_t)n * sizeof(cx<T>);
        ColArgs<T> r = col_base(c);
        r.mode = FIN_RHS;
        r.ko_eta = C(c->ko_eta);
        r.ko_psi = C(c->ko_psi);
        const int save = c->m_run;
        c->m_run = c->M;
        cudaError_t e = rhs(c, C(c->y_eta), C(c->y_psi), r, s, nullptr);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->chk, c->ko_eta, compact, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync((char*)c->chk + compact, c->ko_psi, compact, cudaMemcpyDeviceToDevice, s);
        c->m_run = c->base_M;
        if (e == cudaSuccess) e = rhs(c, C(c->y_eta), C(c->y_psi), r, s, nullptr);
        c->m_run = save;
        if (e == cudaSuccess) e = closure_residual(c, C(c->y_eta), C(c->y_psi), s, nullptr);
        constexpr int nb = 256;
        if (e == cudaSuccess) {
            const double dmax = std::max(c->Lx / c->nx, c->Lz / c->nz);
            closure_err_kernel<T><<<nb, 256, 0, s>>>(C(c->chk), C(c->chk) + n, C(c->ko_eta), C(c->ko_psi), C(c->cspec),
                                                     C(c->cspec) + n, c->nz, c->hx, (T)(2.0 * M_PI / c->Lx),
                                                     (T)(2.0 * M_PI / c->Lz), (T)(2.0 / 3.0 * M_PI / dmax),
                                                     c->opt.taper, c->sc, c->cpart);
            e = cudaGetLastError();
        }
        std::vector<double> hp(2 * nb);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), c->cpart, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return ZK_ECUDA;
        double num = 0.0, den = 0.0;
        for (int i = 0; i < nb; ++i) { num += hp[2 * i]; den += hp[2 * i + 1]; }
        const double err = den > 0.0 ? std::sqrt(num / den) : 0.0;
        c->last_err = err;
        ++c->nchecks;
        if (!(err <= c->check_tol)) {
            c->closure_on = false;
            c->fallback_step = c->nsteps;
            drop_graph(c);
        }
        return ZK_OK;
    }

    // Adaptive order: f_M at the current state, then f_m for m = adapt_min, ...
    // until |f_m - f_M| <= adapt_tol |f_M| (FP64 norms over the spectrum); the
    // context then steps at that order (M if none is within the tolerance).
    static zk_status adapt_check(zk_ctx* c, cudaStream_t s) {
        const long long n = (long long)c->nz * c->hx;
        const size_t compact = (size_t)n * sizeof(cx<T>);
        ColArgs<T> r = col_base(c);
        r.mode = FIN_RHS;
        r.ko_eta = C(c->ko_eta);
        r.ko_psi = C(c->ko_psi);
        const int before = c->m_run;
        c->m_run = c->M;
        cudaError_t e = rhs(c, C(c->y_eta), C(c->y_psi), r, s, nullptr);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->chk, c->ko_eta, compact, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync((char*)c->chk + compact, c->ko_psi, compact, cudaMemcpyDeviceToDevice, s);
        int chosen = c->M;
        for (int m = 0; m <= ZK_MAX_ORDER; ++m) c->adapt_err[m] = -1.0;
        c->adapt_err[c->M] = 0.0;
        constexpr int nb = 256;
        std::vector<double> hp(2 * nb);
        for (int m = c->adapt_min; m < c->M && e == cudaSuccess; ++m) {
            c->m_run = m;
            e = rhs(c, C(c->y_eta), C(c->y_psi), r, s, nullptr);
            if (e != cudaSuccess) break;
            diff_norm_kernel<T><<<nb, 256, 0, s>>>(C(c->chk), C(c->chk) + n, C(c->ko_eta), C(c->ko_psi), c->nz, c->hx,
                                                   c->cpart);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), c->cpart, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) break;
            double num = 0.0, den = 0.0;
            for (int i = 0; i < nb; ++i) { num += hp[2 * i]; den += hp[2 * i + 1]; }
            c->adapt_err[m] = den > 0.0 ? std::sqrt(num / den) : 0.0;
            if (c->adapt_err[m] <= c->adapt_tol) { chosen = m; break; }
        }
        c->m_run = before;
        if (e != cudaSuccess) return ZK_ECUDA;
        ++c->adapt_checks;
        if (chosen != before) {
            c->m_run = chosen;
            c->ab_valid = false;   // IF-AB2 history holds forcing of the old order: restart with IF-Euler
            drop_graph(c);
        }
        return ZK_OK;
    }

    // Training pairs at the current state: features (6 physical channels,
    // divided by in_scale) and, when tgt is non-null, the residual f_M - f_base
    // (2 physical channels, divided by out_scale). Device FP32 outputs.
    static cudaError_t closure_features(zk_ctx* c, float* feat, float* tgt, cudaStream_t s) {
        const long long n = (long long)c->nz * c->hx;
        const size_t compact = (size_t)n * sizeof(cx<T>);
        const size_t plane = (size_t)c->nx * c->nz;
        ColArgs<T> r = col_base(c);
        r.mode = FIN_RHS;
        r.ko_eta = C(c->ko_eta);
        r.ko_psi = C(c->ko_psi);
        const int save = c->m_run;
        cudaError_t e = cudaSuccess;
        if (tgt) {
            c->m_run = c->M;
            e = rhs(c, C(c->y_eta), C(c->y_psi), r, s, nullptr);
            if (e == cudaSuccess) e = cudaMemcpyAsync(c->chk, c->ko_eta, compact, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync((char*)c->chk + compact, c->ko_psi, compact, cudaMemcpyDeviceToDevice, s);
        }
        c->m_run = c->base_M;
        if (e == cudaSuccess) e = rhs(c, C(c->y_eta), C(c->y_psi), r, s, nullptr);
        c->m_run = save;
        cx<T>* cs = C(c->cspec);
        if (e == cudaSuccess && tgt) {
            // the difference kernel reads each pair as one contiguous [eta | psi] block
            e = cudaMemcpyAsync(cs + 2 * n, c->ko_eta, compact, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(cs + 3 * n, c->ko_psi, compact, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) {
                closure_diff_kernel<T><<<4 * 148, 256, 0, s>>>(C(c->chk), cs + 2 * n, cs, n, c->sc);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = to_physical(c, cs, cs + n, tgt, tgt + plane, ZK_F32, s);
        }
        if (e == cudaSuccess) {
            closure_prep_kernel<T><<<4 * 148, 256, 0, s>>>(C(c->y_eta), C(c->y_psi), C(c->ko_eta), C(c->ko_psi), cs, c->nz,
                                                           c->hx, (T)(2.0 * M_PI / c->Lx), (T)(2.0 * M_PI / c->Lz),
                                                           (T)c->h, (T)c->g, c->sc);
            e = cudaGetLastError();
        }
        for (int k = 0; k < 3 && e == cudaSuccess; ++k)
            e = to_physical(c, cs + 2 * k * n, cs + (2 * k + 1) * n, feat + 2 * k * plane, feat + (2 * k + 1) * plane, ZK_F32, s);
        return e;
    }

    // Integrating-factor RK4: four right-hand sides, Lawson stage combination in the epilogue.
    static cudaError_t ifrk4_step(zk_ctx* c, double dt, cudaStream_t s, int* nlaunch) {
        for (int st = 1; st <= 4; ++st) {
            ColArgs<T> fin = col_base(c);
            fin.mode = FIN_IRK1 + st - 1;
            fin.dt = (T)dt;
            fin.y_eta = C(c->y_eta); fin.y_psi = C(c->y_psi);
            fin.ys_eta = C(c->ys_eta); fin.ys_psi = C(c->ys_psi);
            fin.ka_eta = C(c->ka_eta); fin.ka_psi = C(c->ka_psi);
            const cx<T>* se = st == 1 ? C(c->y_eta) : C(c->ys_eta);
            const cx<T>* sp = st == 1 ? C(c->y_psi) : C(c->ys_psi);
            cudaError_t e = rhs(c, se, sp, fin, s, nlaunch);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }

    static cudaError_t ifab2_step(zk_ctx* c, double dt, bool first, cudaStream_t s, int* nlaunch) {
        ColArgs<T> fin = col_base(c);
        fin.mode = FIN_IFAB2;
        fin.dt = (T)dt;
        fin.ab_first = first ? 1 : 0;
        fin.y_eta = C(c->y_eta); fin.y_psi = C(c->y_psi);
        fin.h_eta = C(c->h_eta); fin.h_psi = C(c->h_psi);
        return rhs(c, C(c->y_eta), C(c->y_psi), fin, s, nlaunch);
    }

    // Eq. 19: psi from v_hat at the current eta, `iters` fixed-point updates after psi = v/G0.
    static cudaError_t dno_inverse(zk_ctx* c, const cx<T>* vhat, int iters, cudaStream_t s) {
        const int n = c->nz * c->hx;
        inv_g0_kernel<T><<<(n + 255) / 256, 256, 0, s>>>(vhat, C(c->y_psi), c->nz, c->hx,
                                                         (T)(2.0 * M_PI / c->Lx), (T)(2.0 * M_PI / c->Lz), (T)c->h);
        cudaError_t e = cudaGetLastError();
        for (int it = 0; it < iters && e == cudaSuccess; ++it) {
            ColArgs<T> fin = col_base(c);
            fin.mode = FIN_INVDNO;
            fin.y_psi = C(c->y_psi);
            fin.v_hat = vhat;
            e = rhs(c, C(c->y_eta), C(c->y_psi), fin, s, nullptr);
        }
        return e;
    }

    // Eq. 34 on eta (physical, pointwise), through the ko_psi scratch spectrum.
    static cudaError_t relax_eta(zk_ctx* c, const void* sigma, const void* target, int dtype, double dt,
                                 cudaStream_t s) {
        const cx<T>* twx = reinterpret_cast<const cx<T>*>(c->tw_x);
        const cx<T>* twz = reinterpret_cast<const cx<T>*>(c->tw_z);
        const size_t compact = (size_t)c->nz * c->hx * sizeof(cx<T>);
        cx<T>* f = C(c->ko_psi);
        cudaError_t e = cudaMemcpyAsync(f, c->y_eta, compact, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = launch_cols<T, true>(c->nz, f, nullptr, c->hx, twz, s);
        const T scale = (T)(1.0 / ((double)c->nx * c->nz));
        if (e == cudaSuccess)
            e = dtype == ZK_F32 ? launch_relax_rows<T, float>(c->nx, f, sigma, target, c->nz, (T)dt, scale, twx, s)
                                : launch_relax_rows<T, double>(c->nx, f, sigma, target, c->nz, (T)dt, scale, twx, s);
        if (e == cudaSuccess) e = launch_cols<T, false>(c->nz, f, nullptr, c->hx, twz, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->y_eta, f, compact, cudaMemcpyDeviceToDevice, s);
        return e;
    }

    static cudaError_t rhs_out(zk_ctx* c, cudaStream_t s) {
        ColArgs<T> fin = col_base(c);
        fin.mode = FIN_RHS;
        fin.ko_eta = C(c->ko_eta);
        fin.ko_psi = C(c->ko_psi);
        if (c->closure_on) return closure_stage(c, C(c->y_eta), C(c->y_psi), fin, s, nullptr);
        return rhs(c, C(c->y_eta), C(c->y_psi), fin, s, nullptr);
    }

    static cudaError_t energy(zk_ctx* c, cudaStream_t s) {
        ColArgs<T> fin = col_base(c);
        fin.mode = FIN_ENERGY;
        fin.partial = c->partial;
        cudaError_t e = rhs(c, C(c->y_eta), C(c->y_psi), fin, s, nullptr);
        if (e != cudaSuccess) return e;
        energy_finalize_kernel<<<1, 32, 0, s>>>(c->partial, c->fin_blocks, c->esum);
        return cudaGetLastError();
    }

    // physical [nz][nx] (dtype, device pointer) -> compact state y
    static cudaError_t set_state(zk_ctx* c, const void* de, const void* dp, int dtype, cudaStream_t s) {
        const cx<T>* twx = reinterpret_cast<const cx<T>*>(c->tw_x);
        const cx<T>* twz = reinterpret_cast<const cx<T>*>(c->tw_z);
        cudaError_t e = dtype == ZK_F32
            ? launch_rows_fwd<T, float>(c->nx, de, dp, c->nz, C(c->y_eta), C(c->y_psi), twx, s)
            : launch_rows_fwd<T, double>(c->nx, de, dp, c->nz, C(c->y_eta), C(c->y_psi), twx, s);
        if (e != cudaSuccess) return e;
        return launch_cols<T, false>(c->nz, C(c->y_eta), C(c->y_psi), c->hx, twz, s);
    }

    // compact (a, b) -> physical (dtype, device pointers); a, b are overwritten
    static cudaError_t to_physical(zk_ctx* c, cx<T>* a, cx<T>* b, void* oa, void* ob, int dtype, cudaStream_t s) {
        const cx<T>* twx = reinterpret_cast<const cx<T>*>(c->tw_x);
        const cx<T>* twz = reinterpret_cast<const cx<T>*>(c->tw_z);
        cudaError_t e = launch_cols<T, true>(c->nz, a, b, c->hx, twz, s);
        if (e != cudaSuccess) return e;
        const T scale = (T)(1.0 / ((double)c->nx * c->nz));
        return dtype == ZK_F32
            ? launch_rows_inv<T, float>(c->nx, a, b, c->nz, scale, oa, ob, twx, s)
            : launch_rows_inv<T, double>(c->nx, a, b, c->nz, scale, oa, ob, twx, s);
    }
};

// Stockham tables (length-n w_n^t) for the unpadded state transforms; per-stage
// tables of the in-place plans for the padded right-hand-side transforms.
template <typename T>
void make_plan_twiddles(int n, int v, std::vector<cx<T>>& out) {
    const PlanDesc d = plan_desc_of(n, v);
    const int ne = plan_table_size(d);
    out.resize(ne);
    for (int e = 0; e < ne; ++e) {
        long long num;
        int den;
        plan_table_entry(d, e, &num, &den);
        const double ang = -2.0 * M_PI * (double)num / (double)den;
        out[e] = mk<T>((T)std::cos(ang), (T)std::sin(ang));
    }
}

template <typename T>
zk_status upload(zk_ctx* c, const std::vector<cx<T>>& h, void** dst) {
    void* p = nullptr;
    if (cudaMalloc(&p, h.size() * sizeof(cx<T>)) != cudaSuccess) { cudaGetLastError(); return ZK_ENOMEM; }
    c->allocs.push_back(p);
    c->bytes += h.size() * sizeof(cx<T>);
    if (cudaMemcpy(p, h.data(), h.size() * sizeof(cx<T>), cudaMemcpyHostToDevice) != cudaSuccess) return ZK_ECUDA;
    *dst = p;
    return ZK_OK;
}

template <typename T>
zk_status alloc_twiddles(zk_ctx* c) {
    std::vector<cx<T>> h;
    make_twiddles<T>(c->nx, h);
    zk_status st = upload<T>(c, h, &c->tw_x);
    if (st == ZK_OK) { make_twiddles<T>(c->nz, h); st = upload<T>(c, h, &c->tw_z); }
    const int np[2] = {c->npx, c->npz};
    for (int v = 0; v < 2 && st == ZK_OK; ++v) {
        for (int i = 0; i < 2 && st == ZK_OK; ++i) {
            if (v == 1 && !plan_has_variant(np[i])) { c->tw_pv[1][i] = c->tw_pv[0][i]; continue; }
            make_plan_twiddles<T>(np[i], v, h);
            st = upload<T>(c, h, &c->tw_pv[v][i]);
        }
    }
    c->tw_px = c->tw_pv[0][0];
    c->tw_pz = c->tw_pv[0][1];
    bool any_half = false;
    for (int v = 0; v < 2 && st == ZK_OK; ++v) {
        if (!half_plan_ok_host(c->npx, v)) continue;
        make_plan_twiddles<T>(c->npx / 2, v, h);
        st = upload<T>(c, h, &c->tw_hv[v]);
        any_half = true;
    }
    if (st == ZK_OK && any_half) {
        h.resize(c->npx / 2);
        for (int k = 0; k < c->npx / 2; ++k) {
            const double ang = -2.0 * M_PI * (double)k / (double)c->npx;
            h[k] = mk<T>((T)std::cos(ang), (T)std::sin(ang));
        }
        st = upload<T>(c, h, &c->tw_rx);
    }
    return st;
}

zk_status dalloc(zk_ctx* c, void** p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) { *p = nullptr; cudaGetLastError(); return ZK_ENOMEM; }
    c->allocs.push_back(*p);
    c->bytes += bytes;
    if (cudaMemset(*p, 0, bytes) != cudaSuccess) return ZK_ECUDA;
    return ZK_OK;
}

void drop_graph(zk_ctx* c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->gexec_boot) cudaGraphExecDestroy(c->gexec_boot);
    c->gexec = nullptr;
    c->gexec_boot = nullptr;
    c->gvalid = false;
}

// variant: 0 = RK4 step, 1 = IF-AB2 bootstrap step, 2 = IF-AB2 step with history
cudaError_t enqueue_step_any(zk_ctx* c, double dt, cudaStream_t s, int* nl, int variant) {
    if (variant == 0) {
        if (c->opt.integrator == ZK_IFRK4)
            return c->prec == ZK_F32 ? Pipe<float>::ifrk4_step(c, dt, s, nl) : Pipe<double>::ifrk4_step(c, dt, s, nl);
        if (c->closure_on && c->prec == ZK_F32) return Pipe<float>::closure_rk4_step(c, dt, s, nl);
        return c->prec == ZK_F32 ? Pipe<float>::rk4_step(c, dt, s, nl) : Pipe<double>::rk4_step(c, dt, s, nl);
    }
    const bool first = variant == 1;
    return c->prec == ZK_F32 ? Pipe<float>::ifab2_step(c, dt, first, s, nl)
                             : Pipe<double>::ifab2_step(c, dt, first, s, nl);
}

zk_status capture(zk_ctx* c, double dt, int variant, cudaGraphExec_t* out, int* nl) {
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) return ZK_ECUDA;
    cudaError_t e = enqueue_step_any(c, dt, c->cap, nl, variant);
    cudaError_t e2 = cudaStreamEndCapture(c->cap, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return ZK_ECUDA;
    }
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { *out = nullptr; return ZK_ECUDA; }
    return ZK_OK;
}

zk_status build_graph(zk_ctx* c, double dt) {
    drop_graph(c);
    if (!c->cap) {
        if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) return ZK_ECUDA;
    }
    int nl = 0;
    zk_status st;
    if (c->opt.integrator == ZK_IFAB2) {
        st = capture(c, dt, 1, &c->gexec_boot, &nl);
        if (st != ZK_OK) return st;
        nl = 0;
        st = capture(c, dt, 2, &c->gexec, &nl);
    } else {
        st = capture(c, dt, 0, &c->gexec, &nl);
    }
    if (st != ZK_OK) { drop_graph(c); return st; }
    c->gvalid = true;
    c->gdt = dt;
    c->launches_per_step = nl;
    return ZK_OK;
}

// Copy helpers between caller buffers and the staging area.
zk_status stage_in(zk_ctx* c, const void* a, const void* b, int dtype, int on_device, const void** da, const void** db) {
    const size_t n = (size_t)c->nx * c->nz * (dtype == ZK_F32 ? 4 : 8);
    if (on_device) { *da = a; *db = b; return ZK_OK; }
    char* st = (char*)c->stage;
    cudaStream_t s = user_stream(c);
    if (cudaMemcpyAsync(st, a, n, cudaMemcpyHostToDevice, s) != cudaSuccess) return ZK_ECUDA;
    if (cudaMemcpyAsync(st + (size_t)c->nx * c->nz * kIoElem, b, n, cudaMemcpyHostToDevice, s) != cudaSuccess) return ZK_ECUDA;
    *da = st;
    *db = st + (size_t)c->nx * c->nz * kIoElem;
    return ZK_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* zk_strerror(zk_status s) {
    switch (s) {
    case ZK_OK: return "ok";
    case ZK_EINVAL: return "invalid argument";
    case ZK_ENOMEM: return "out of memory";
    case ZK_ECUDA: return "CUDA error";
    case ZK_ENONFINITE: return "state is not finite";
    case ZK_ETIMEOUT: return "device wait timed out";
    case ZK_EUNSUPPORTED: return "unsupported";
    case ZK_ESTATE: return "call out of order";
    default: return "unknown status";
    }
}

const char* zk_version(void) { return "zk 0.1 sm_103a"; }

void zk_destroy(zk_ctx* c) {
    if (!c) return;
    drop_graph(c);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->io) {
        cudaStreamSynchronize(c->io);
        cudaStreamSynchronize(c->io_out);
        cudaStreamDestroy(c->io);
        cudaStreamDestroy(c->io_out);
        for (int k = 0; k < 2; ++k) {
            cudaEventDestroy(c->ev_in[k]); cudaEventDestroy(c->ev_in_used[k]);
            cudaEventDestroy(c->ev_out[k]); cudaEventDestroy(c->ev_out_done[k]);
        }
    }
    for (void* p : c->allocs) cudaFree(p);
    delete c;
}

}  // extern "C"

namespace {

// One context over nb tiles of the same grid and order with depths h[0..nb-1].
zk_status ctx_create(zk_ctx** out, int nx, int nz, double Lx, double Lz, const double* h, int nb, double g, int M,
                     int precision, int pad3 = 0) {
    if (!out || !h || nb < 1) return ZK_EINVAL;
    *out = nullptr;
    if (!is_pow2(nx) || !is_pow2(nz) || nx < 16 || nz < 16) return ZK_EINVAL;
    const int nmax = precision == ZK_F64 ? 1024 : 2048;
    if (nx > nmax || nz > nmax) return ZK_EINVAL;
    if (!(Lx > 0) || !(Lz > 0) || !(g > 0)) return ZK_EINVAL;
    for (int t = 0; t < nb; ++t) if (!(h[t] > 0)) return ZK_EINVAL;
    if (M < 1 || M > ZK_MAX_ORDER) return ZK_EINVAL;
    if (precision != ZK_F32 && precision != ZK_F64) return ZK_EINVAL;
    zk_ctx* c = new (std::nothrow) zk_ctx();
    if (!c) return ZK_ENOMEM;
    if (pad3 && (precision != ZK_F32 || nx > 1024 || nz > 1024)) { delete c; return ZK_EUNSUPPORTED; }
    c->pad3 = pad3 != 0;
    c->nx = nx; c->nz = nz; c->hx = nx / 2;
    c->npx = pad3 ? 3 * nx : 3 * nx / 2;
    c->npz = pad3 ? 3 * nz : 3 * nz / 2;
    c->Lx = Lx; c->Lz = Lz; c->h = h[0]; c->g = g; c->M = M; c->m_run = M; c->prec = precision;
    c->opt.eps = 1.0; c->opt.integrator = ZK_RK4; c->opt.taper = 1; c->opt.filter = 1; c->opt.stream = nullptr;
    c->nb = nb;
    c->hv.assign(h, h + nb);
    cudaGetDevice(&c->device);
    c->csz = precision == ZK_F32 ? 8 : 16;
    const size_t rsz = precision == ZK_F32 ? 4 : 8;
    zk_status st = precision == ZK_F32 ? alloc_twiddles<float>(c) : alloc_twiddles<double>(c);
    c->tst = (long long)nz * c->hx;
    const size_t compact = (size_t)c->tst * c->csz * nb;
    void** comp[10] = {&c->y_eta, &c->y_psi, &c->ys_eta, &c->ys_psi, &c->ka_eta, &c->ka_psi,
                       &c->ko_eta, &c->ko_psi, &c->h_eta, &c->h_psi};
    for (int i = 0; i < 10 && st == ZK_OK; ++i) st = dalloc(c, comp[i], compact);
    const Fields F{M};
    c->nfields = F.count();
    c->fstride = (long long)c->npz * c->hx;
    c->tcol = (long long)c->nfields * c->fstride;
    c->tacc = (long long)c->npz * c->npx;
    if (st == ZK_OK) st = dalloc(c, &c->col, (size_t)c->tcol * c->csz * nb);
    // 8 bytes per element in every precision, so FP32 contexts can switch on FP64 series sums
    if (st == ZK_OK) st = dalloc(c, &c->acc, (size_t)c->tacc * 8 * nb);
    if (st == ZK_OK && M >= 2) st = dalloc(c, &c->sfc, (size_t)3 * c->tacc * rsz * nb);
    if (st == ZK_OK && c->npz >= 1536) st = dalloc(c, &c->fsc, 2 * compact);
    if (st == ZK_OK) st = dalloc(c, &c->stage, (size_t)2 * nx * nz * kIoElem);
    if (st == ZK_OK) st = dalloc(c, &c->tank, (size_t)2 * (nx / 2) * (nz / 2) * 8);
    c->npartial = c->hx * nb;              // at most one column-kernel block per column
    if (st == ZK_OK) st = dalloc(c, (void**)&c->partial, (size_t)3 * c->npartial * sizeof(double));
    if (st == ZK_OK) st = dalloc(c, (void**)&c->esum, 4 * sizeof(double));
    if (st == ZK_OK && nb > 1) {
        st = dalloc(c, &c->hb, (size_t)nb * rsz);
        if (st == ZK_OK) {
            std::vector<float> hf(h, h + nb);
            const void* src = precision == ZK_F32 ? (const void*)hf.data() : (const void*)h;
            if (cudaMemcpy(c->hb, src, (size_t)nb * rsz, cudaMemcpyHostToDevice) != cudaSuccess) st = ZK_ECUDA;
        }
    }
    if (st != ZK_OK) { zk_destroy(c); return st; }
    *out = c;
    return ZK_OK;
}

// Single-tile view of tile t of a group context: the same buffers offset to the
// tile, depth h[t]; owns nothing (never destroyed), has no graph.
void tile_view(const zk_ctx* g, int t, zk_ctx* v) {
    v->nx = g->nx; v->nz = g->nz; v->npx = g->npx; v->npz = g->npz; v->hx = g->hx; v->M = g->M; v->prec = g->prec;
    v->Lx = g->Lx; v->Lz = g->Lz; v->h = g->hv[t]; v->g = g->g;
    v->opt = g->opt;
    v->device = g->device;
    v->has_state = true;
    v->csz = g->csz;
    v->tw_x = g->tw_x; v->tw_z = g->tw_z; v->tw_px = g->tw_px; v->tw_pz = g->tw_pz;
    v->tw_pv[0][0] = g->tw_pv[0][0]; v->tw_pv[0][1] = g->tw_pv[0][1];
    v->tw_pv[1][0] = g->tw_pv[1][0]; v->tw_pv[1][1] = g->tw_pv[1][1];
    v->tw_hv[0] = g->tw_hv[0]; v->tw_hv[1] = g->tw_hv[1]; v->tw_rx = g->tw_rx;
    const size_t oc = (size_t)t * g->tst * g->csz;
    auto off = [&](void* p, size_t o) { return p ? (void*)((char*)p + o) : nullptr; };
    v->y_eta = off(g->y_eta, oc); v->y_psi = off(g->y_psi, oc);
    v->ys_eta = off(g->ys_eta, oc); v->ys_psi = off(g->ys_psi, oc);
    v->ka_eta = off(g->ka_eta, oc); v->ka_psi = off(g->ka_psi, oc);
    v->ko_eta = off(g->ko_eta, oc); v->ko_psi = off(g->ko_psi, oc);
    v->h_eta = off(g->h_eta, oc); v->h_psi = off(g->h_psi, oc);
    v->col = off(g->col, (size_t)t * g->tcol * g->csz);
    v->acc = off(g->acc, (size_t)t * g->tacc * ((g->prec == ZK_F32 && !g->series64) ? 4 : 8));
    v->sfc = off(g->sfc, (size_t)t * 3 * g->tacc * (g->prec == ZK_F32 ? 4 : 8));
    v->series64 = g->series64;
    v->pad3 = g->pad3;
    v->nfields = g->nfields;
    v->fstride = g->fstride;
    v->stage = g->stage; v->tank = g->tank;
    v->partial = g->partial; v->npartial = g->npartial; v->esum = g->esum;
    v->nb = 1; v->tcol = 0; v->tst = 0; v->tacc = 0; v->hb = nullptr;
    v->hv.assign(1, g->hv[t]);
    v->plan_v = g->plan_v; v->col_ci = g->col_ci; v->row_occ = g->row_occ;
}

}  // namespace

extern "C" {

zk_status zk_create(zk_ctx** out, int nx, int nz, double Lx, double Lz, double h, double g, int M, int precision) {
    return ctx_create(out, nx, nz, Lx, Lz, &h, 1, g, M, precision);
}

zk_status zk_create_ex(zk_ctx** out, int nx, int nz, double Lx, double Lz, double h, double g, int M, int precision,
                       int pad) {
    if (pad != ZK_PAD_3_2 && pad != ZK_PAD_3) {
        if (out) *out = nullptr;
        return ZK_EINVAL;
    }
    return ctx_create(out, nx, nz, Lx, Lz, &h, 1, g, M, precision, pad == ZK_PAD_3 ? 1 : 0);
}

zk_status zk_set_options(zk_ctx* c, const zk_options* o) {
    if (!c || !o) return ZK_EINVAL;
    if (!(o->eps >= 0.0 && o->eps <= 1.0)) return ZK_EINVAL;
    if (o->integrator != ZK_RK4 && o->integrator != ZK_IFAB2 && o->integrator != ZK_IFRK4) return ZK_EINVAL;
    if ((o->taper != 0 && o->taper != 1) || (o->filter != 0 && o->filter != 1)) return ZK_EINVAL;
    if (o->integrator != c->opt.integrator || o->eps != c->opt.eps || o->taper != c->opt.taper)
        c->ab_valid = false;   // the forcing history belongs to the old right-hand side
    c->opt = *o;
    drop_graph(c);
    return ZK_OK;
}

zk_status zk_get_options(const zk_ctx* c, zk_options* o) {
    if (!c || !o) return ZK_EINVAL;
    *o = c->opt;
    return ZK_OK;
}

zk_status zk_set_state(zk_ctx* c, const void* eta, const void* psi, int dtype, int on_device) {
    if (!c || !eta || !psi || (dtype != ZK_F32 && dtype != ZK_F64)) return ZK_EINVAL;
    const void *de, *dp;
    zk_status st = stage_in(c, eta, psi, dtype, on_device, &de, &dp);
    if (st != ZK_OK) return st;
    cudaError_t e = c->prec == ZK_F32 ? Pipe<float>::set_state(c, de, dp, dtype, user_stream(c))
                                      : Pipe<double>::set_state(c, de, dp, dtype, user_stream(c));
    if (e != cudaSuccess) return ZK_ECUDA;
    c->has_state = true;
    c->ab_valid = false;
    return ZK_OK;
}

static zk_status out_physical(zk_ctx* c, void* ca, void* cb, void* oa, void* ob, int dtype, int on_device) {
    cudaStream_t s = user_stream(c);
    const size_t n = (size_t)c->nx * c->nz * (dtype == ZK_F32 ? 4 : 8);
    char* st = (char*)c->stage;
    void* da = on_device ? oa : (void*)st;
    void* db = ob ? (on_device ? ob : (void*)(st + (size_t)c->nx * c->nz * kIoElem)) : nullptr;
    cudaError_t e = c->prec == ZK_F32
        ? Pipe<float>::to_physical(c, (cx<float>*)ca, (cx<float>*)cb, da, db, dtype, s)
        : Pipe<double>::to_physical(c, (cx<double>*)ca, (cx<double>*)cb, da, db, dtype, s);
    if (e != cudaSuccess) return ZK_ECUDA;
    if (!on_device) {
        if (cudaMemcpyAsync(oa, da, n, cudaMemcpyDeviceToHost, s) != cudaSuccess) return ZK_ECUDA;
        if (ob && cudaMemcpyAsync(ob, db, n, cudaMemcpyDeviceToHost, s) != cudaSuccess) return ZK_ECUDA;
    }
    return cu(cudaStreamSynchronize(s));
}

zk_status zk_get_state(zk_ctx* c, void* eta, void* psi, int dtype, int on_device) {
    if (!c || !eta || (dtype != ZK_F32 && dtype != ZK_F64)) return ZK_EINVAL;
    if (!c->has_state) return ZK_ESTATE;
    cudaStream_t s = user_stream(c);
    const size_t compact = (size_t)c->nz * c->hx * c->csz;
    if (cudaMemcpyAsync(c->ko_eta, c->y_eta, compact, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return ZK_ECUDA;
    if (cudaMemcpyAsync(c->ko_psi, c->y_psi, compact, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return ZK_ECUDA;
    return out_physical(c, c->ko_eta, c->ko_psi, eta, psi, dtype, on_device);
}

zk_status zk_rhs(zk_ctx* c, void* deta, void* dpsi, int dtype, int on_device) {
    if (!c || !deta || (dtype != ZK_F32 && dtype != ZK_F64)) return ZK_EINVAL;
    if (!c->has_state) return ZK_ESTATE;
    cudaError_t e = c->prec == ZK_F32 ? Pipe<float>::rhs_out(c, user_stream(c)) : Pipe<double>::rhs_out(c, user_stream(c));
    if (e != cudaSuccess) return ZK_ECUDA;
    return out_physical(c, c->ko_eta, c->ko_psi, deta, dpsi, dtype, on_device);
}

zk_status zk_dno(zk_ctx* c, void* v, int dtype, int on_device) {
    if (!c || !v || (dtype != ZK_F32 && dtype != ZK_F64)) return ZK_EINVAL;
    if (!c->has_state) return ZK_ESTATE;
    cudaError_t e = c->prec == ZK_F32 ? Pipe<float>::rhs_out(c, user_stream(c)) : Pipe<double>::rhs_out(c, user_stream(c));
    if (e != cudaSuccess) return ZK_ECUDA;
    return out_physical(c, c->ko_eta, nullptr, v, nullptr, dtype, on_device);
}

// Tank (walled) I/O through the even extension (Sec. 3.3): the context's grid is
// the doubled one; the caller's arrays are the (nx/2) x (nz/2) tank. Tank copies
// go to their own buffer (c->tank, two FP64-sized tank arrays); the extended
// fields go to the two staging slots, so no copy overlaps another.
zk_status zk_set_state_tank(zk_ctx* c, const void* eta, const void* psi, int dtype, int on_device) {
    if (!c || !eta || !psi || (dtype != ZK_F32 && dtype != ZK_F64)) return ZK_EINVAL;
    const int mx = c->nx / 2, mz = c->nz / 2;
    const size_t es = dtype == ZK_F32 ? 4 : 8, tank = (size_t)mx * mz * es;
    cudaStream_t s = user_stream(c);
    char* te = (char*)c->tank;
    char* tp = te + (size_t)mx * mz * 8;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (cudaMemcpyAsync(te, eta, tank, k, s) != cudaSuccess) return ZK_ECUDA;
    if (cudaMemcpyAsync(tp, psi, tank, k, s) != cudaSuccess) return ZK_ECUDA;
    char* de = (char*)c->stage;
    char* dp = de + (size_t)c->nx * c->nz * kIoElem;
    const int blocks = 4 * 148, threads = 256;
    if (dtype == ZK_F32) {
        even_extend_kernel<float><<<blocks, threads, 0, s>>>((const float*)te, (float*)de, mx, mz);
        even_extend_kernel<float><<<blocks, threads, 0, s>>>((const float*)tp, (float*)dp, mx, mz);
    } else {
        even_extend_kernel<double><<<blocks, threads, 0, s>>>((const double*)te, (double*)de, mx, mz);
        even_extend_kernel<double><<<blocks, threads, 0, s>>>((const double*)tp, (double*)dp, mx, mz);
    }
    if (cudaGetLastError() != cudaSuccess) return ZK_ECUDA;
    return zk_set_state(c, de, dp, dtype, 1);
}

zk_status zk_get_state_tank(zk_ctx* c, void* eta, void* psi, int dtype, int on_device) {
    if (!c || !eta || !psi || (dtype != ZK_F32 && dtype != ZK_F64)) return ZK_EINVAL;
    if (!c->has_state) return ZK_ESTATE;
    const int mx = c->nx / 2, mz = c->nz / 2;
    const size_t es = dtype == ZK_F32 ? 4 : 8;
    cudaStream_t s = user_stream(c);
    char* fe = (char*)c->stage;                                 // full doubled fields, device
    char* fp = fe + (size_t)c->nx * c->nz * kIoElem;
    zk_status r = zk_get_state(c, fe, fp, dtype, 1);
    if (r != ZK_OK) return r;
    if (on_device) {
        const int blocks = 148, threads = 256;
        if (dtype == ZK_F32) {
            crop_kernel<float><<<blocks, threads, 0, s>>>((const float*)fe, (float*)eta, mx, mz);
            crop_kernel<float><<<blocks, threads, 0, s>>>((const float*)fp, (float*)psi, mx, mz);
        } else {
            crop_kernel<double><<<blocks, threads, 0, s>>>((const double*)fe, (double*)eta, mx, mz);
            crop_kernel<double><<<blocks, threads, 0, s>>>((const double*)fp, (double*)psi, mx, mz);
        }
        if (cudaGetLastError() != cudaSuccess) return ZK_ECUDA;
    } else {
        const size_t row = (size_t)mx * es, pitch = (size_t)2 * mx * es;
        if (cudaMemcpy2DAsync(eta, row, fe, pitch, row, mz, cudaMemcpyDeviceToHost, s) != cudaSuccess) return ZK_ECUDA;
        if (cudaMemcpy2DAsync(psi, row, fp, pitch, row, mz, cudaMemcpyDeviceToHost, s) != cudaSuccess) return ZK_ECUDA;
    }
    return cu(cudaStreamSynchronize(s));
}

zk_status zk_dno_inverse(zk_ctx* c, const void* v, int dtype, int on_device, int iters) {
    if (!c || !v || (dtype != ZK_F32 && dtype != ZK_F64) || iters < 0) return ZK_EINVAL;
    if (!c->has_state) return ZK_ESTATE;
    const void *dv, *dv2;
    zk_status st = stage_in(c, v, v, dtype, on_device, &dv, &dv2);
    if (st != ZK_OK) return st;
    cudaStream_t s = user_stream(c);
    cudaError_t e;
    if (c->prec == ZK_F32) {
        auto* ve = (cx<float>*)c->ko_eta;
        e = dtype == ZK_F32
            ? launch_rows_fwd<float, float>(c->nx, dv, dv, c->nz, ve, (cx<float>*)c->ko_psi, (const cx<float>*)c->tw_x, s)
            : launch_rows_fwd<float, double>(c->nx, dv, dv, c->nz, ve, (cx<float>*)c->ko_psi, (const cx<float>*)c->tw_x, s);
        if (e == cudaSuccess) e = launch_cols<float, false>(c->nz, ve, nullptr, c->hx, (const cx<float>*)c->tw_z, s);
        if (e == cudaSuccess) e = Pipe<float>::dno_inverse(c, ve, iters, s);
    } else {
        auto* ve = (cx<double>*)c->ko_eta;
        e = dtype == ZK_F32
            ? launch_rows_fwd<double, float>(c->nx, dv, dv, c->nz, ve, (cx<double>*)c->ko_psi, (const cx<double>*)c->tw_x, s)
            : launch_rows_fwd<double, double>(c->nx, dv, dv, c->nz, ve, (cx<double>*)c->ko_psi, (const cx<double>*)c->tw_x, s);
        if (e == cudaSuccess) e = launch_cols<double, false>(c->nz, ve, nullptr, c->hx, (const cx<double>*)c->tw_z, s);
        if (e == cudaSuccess) e = Pipe<double>::dno_inverse(c, ve, iters, s);
    }
    if (e != cudaSuccess) return ZK_ECUDA;
    return cu(cudaStreamSynchronize(s));
}

zk_status zk_relax(zk_ctx* c, const void* sigma, const void* eta_target, int dtype, int on_device, double dt, int iters) {
    if (!c || !sigma || !eta_target || (dtype != ZK_F32 && dtype != ZK_F64) || iters < 0 || !(dt >= 0)) return ZK_EINVAL;
    if (!c->has_state) return ZK_ESTATE;
    const void *ds, *dtg;
    zk_status st = stage_in(c, sigma, eta_target, dtype, on_device, &ds, &dtg);
    if (st != ZK_OK) return st;
    cudaStream_t s = user_stream(c);
    cudaError_t e;
    if (c->prec == ZK_F32) {
        e = Pipe<float>::rhs_out(c, s);                                  // v = G(eta) psi into ko_eta
        if (e == cudaSuccess) e = Pipe<float>::relax_eta(c, ds, dtg, dtype, dt, s);
        if (e == cudaSuccess) e = Pipe<float>::dno_inverse(c, (const cx<float>*)c->ko_eta, iters, s);
    } else {
        e = Pipe<double>::rhs_out(c, s);
        if (e == cudaSuccess) e = Pipe<double>::relax_eta(c, ds, dtg, dtype, dt, s);
        if (e == cudaSuccess) e = Pipe<double>::dno_inverse(c, (const cx<double>*)c->ko_eta, iters, s);
    }
    if (e != cudaSuccess) return ZK_ECUDA;
    return cu(cudaStreamSynchronize(s));
}

zk_status zk_step(zk_ctx* c, double dt, int n) {
    if (!c || n < 0 || !(dt > 0) || !std::isfinite(dt)) return ZK_EINVAL;
    if (!c->has_state) return ZK_ESTATE;
    if (c->closure_on && c->opt.integrator != ZK_RK4) return ZK_EUNSUPPORTED;
    cudaStream_t s = user_stream(c);
    for (int i = 0; i < n; ++i) {
        if (c->adapt_every > 0 && c->nsteps % c->adapt_every == 0) {
            zk_status st = c->prec == ZK_F32 ? Pipe<float>::adapt_check(c, s) : Pipe<double>::adapt_check(c, s);
            if (st != ZK_OK) return st;
        }
        if (c->closure_on && c->check_every > 0 && c->nsteps % c->check_every == 0) {
            zk_status st = Pipe<float>::closure_check(c, s);   // may switch the closure off
            if (st != ZK_OK) return st;
        }
        if (!c->gvalid || c->gdt != dt) {
            zk_status st = build_graph(c, dt);
            if (st != ZK_OK) return st;
        }
        cudaGraphExec_t g = c->gexec;
        if (c->opt.integrator == ZK_IFAB2 && !(c->ab_valid && c->ab_dt == dt)) {
            // first step, or a step whose dt differs from the history's: IF-Euler (Sec. 3.4)
            g = c->gexec_boot;
            c->ab_valid = true;
            c->ab_dt = dt;
        }
        if (cudaGraphLaunch(g, s) != cudaSuccess) return ZK_ECUDA;
        ++c->nsteps;
    }
    return ZK_OK;
}

zk_status zk_energy(zk_ctx* c, double* H, double* kin, double* pot, double* mean_eta) {
    if (!c) return ZK_EINVAL;
    if (!c->has_state) return ZK_ESTATE;
    cudaStream_t s = user_stream(c);
    cudaError_t e = c->prec == ZK_F32 ? Pipe<float>::energy(c, s) : Pipe<double>::energy(c, s);
    if (e != cudaSuccess) return ZK_ECUDA;
    double hs[3];
    if (cudaMemcpyAsync(hs, c->esum, sizeof(hs), cudaMemcpyDeviceToHost, s) != cudaSuccess) return ZK_ECUDA;
    double m0[2] = {0, 0};
    if (c->prec == ZK_F32) {
        float2 v;
        if (cudaMemcpyAsync(&v, c->y_eta, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess) return ZK_ECUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return ZK_ECUDA;
        m0[0] = v.x;
    } else {
        double2 v;
        if (cudaMemcpyAsync(&v, c->y_eta, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess) return ZK_ECUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return ZK_ECUDA;
        m0[0] = v.x;
    }
    const double nn = (double)c->nx * c->nz;
    const double w = (c->Lx / c->nx) * (c->Lz / c->nz) / nn;
    const double k = 0.5 * w * hs[0];
    const double p = 0.5 * c->g * w * hs[1];
    if (H) *H = k + p;
    if (kin) *kin = k;
    if (pot) *pot = p;
    if (mean_eta) *mean_eta = m0[0] / nn;
    if (hs[2] != 0.0 || !std::isfinite(k) || !std::isfinite(p)) return ZK_ENONFINITE;
    return ZK_OK;
}

zk_status zk_profile_step(zk_ctx* c, double dt, int nsteps, double* ms, int* kind, double* bytes, int cap, int* nslots) {
    if (!c || !ms || !nslots || nsteps < 1 || !(dt > 0)) return ZK_EINVAL;
    if (!c->has_state) return ZK_ESTATE;
    cudaStream_t s = user_stream(c);
    int n0 = -1;
    for (int i = 0; i < nsteps; ++i) {
        std::vector<cudaEvent_t> ev;
        c->prof_ev = &ev;
        c->slot_kind.clear();
        c->slot_bytes.clear();
        int nl = 0;
        int variant = 0;
        if (c->opt.integrator == ZK_IFAB2) {
            variant = (c->ab_valid && c->ab_dt == dt) ? 2 : 1;
            c->ab_valid = true;
            c->ab_dt = dt;
        }
        cudaError_t e = enqueue_step_any(c, dt, s, &nl, variant);
        cudaEvent_t last;
        cudaEventCreate(&last);
        cudaEventRecord(last, s);
        ev.push_back(last);
        c->prof_ev = nullptr;
        zk_status st = e == cudaSuccess ? cu(cudaStreamSynchronize(s)) : ZK_ECUDA;
        const int n = (int)ev.size() - 1;
        if (st == ZK_OK) {
            if (n0 < 0) {
                n0 = n;
                if (n > cap) st = ZK_EINVAL;
                else for (int k = 0; k < n; ++k) ms[k] = 0.0;
            }
            if (st == ZK_OK && n == n0) {
                for (int k = 0; k < n; ++k) {
                    float t = 0.f;
                    cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
                    ms[k] += t;
                    if (kind) kind[k] = c->slot_kind[k];
                    if (bytes) bytes[k] = c->slot_bytes[k];
                }
            }
        }
        for (cudaEvent_t x : ev) cudaEventDestroy(x);
        if (st != ZK_OK) return st;
    }
    *nslots = n0;
    return ZK_OK;
}

zk_status zk_sync(zk_ctx* c) {
    if (!c) return ZK_EINVAL;
    if (c->io && (cudaStreamSynchronize(c->io) != cudaSuccess || cudaStreamSynchronize(c->io_out) != cudaSuccess))
        return ZK_ECUDA;
    return cu(cudaStreamSynchronize(user_stream(c)));
}

static zk_status async_io_setup(zk_ctx* c) {
    if (c->io) return ZK_OK;
    const size_t slot = (size_t)2 * c->nx * c->nz * kIoElem;
    zk_status st = ZK_OK;
    for (int k = 0; k < 2 && st == ZK_OK; ++k) {
        st = dalloc(c, &c->astage_in[k], slot);
        if (st == ZK_OK) st = dalloc(c, &c->astage_out[k], slot);
    }
    if (st != ZK_OK) return st;
    for (int k = 0; k < 2; ++k) {
        cudaEvent_t* ev[4] = {&c->ev_in[k], &c->ev_in_used[k], &c->ev_out[k], &c->ev_out_done[k]};
        for (cudaEvent_t* e : ev)
            if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return ZK_ECUDA;
    }
    if (cudaStreamCreateWithFlags(&c->io_out, cudaStreamNonBlocking) != cudaSuccess) { c->io_out = nullptr; return ZK_ECUDA; }
    if (cudaStreamCreateWithFlags(&c->io, cudaStreamNonBlocking) != cudaSuccess) {
        cudaStreamDestroy(c->io_out);
        c->io = c->io_out = nullptr;
        return ZK_ECUDA;
    }
    return ZK_OK;
}

zk_status zk_set_state_async(zk_ctx* c, const void* eta, const void* psi, int dtype) {
    if (!c || !eta || !psi || (dtype != ZK_F32 && dtype != ZK_F64)) return ZK_EINVAL;
    zk_status st = async_io_setup(c);
    if (st != ZK_OK) return st;
    const int k = c->in_slot;
    c->in_slot ^= 1;
    cudaStream_t s = user_stream(c);
    const size_t n = (size_t)c->nx * c->nz * (dtype == ZK_F32 ? 4 : 8);
    char* a = (char*)c->astage_in[k];
    char* b = a + (size_t)c->nx * c->nz * kIoElem;
    cudaError_t e = cudaSuccess;
    if (c->in_used_rec[k]) e = cudaStreamWaitEvent(c->io, c->ev_in_used[k], 0);   // the slot's last reader is done
    if (e == cudaSuccess) e = cudaMemcpyAsync(a, eta, n, cudaMemcpyHostToDevice, c->io);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b, psi, n, cudaMemcpyHostToDevice, c->io);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_in[k], c->io);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->ev_in[k], 0);
    if (e == cudaSuccess)
        e = c->prec == ZK_F32 ? Pipe<float>::set_state(c, a, b, dtype, s) : Pipe<double>::set_state(c, a, b, dtype, s);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_in_used[k], s);
    if (e != cudaSuccess) return ZK_ECUDA;
    c->in_used_rec[k] = true;
    c->has_state = true;
    c->ab_valid = false;
    return ZK_OK;
}

zk_status zk_get_state_async(zk_ctx* c, void* eta, void* psi, int dtype) {
    if (!c || !eta || !psi || (dtype != ZK_F32 && dtype != ZK_F64)) return ZK_EINVAL;
    if (!c->has_state) return ZK_ESTATE;
    zk_status st = async_io_setup(c);
    if (st != ZK_OK) return st;
    const int k = c->out_slot;
    c->out_slot ^= 1;
    cudaStream_t s = user_stream(c);
    const size_t n = (size_t)c->nx * c->nz * (dtype == ZK_F32 ? 4 : 8);
    const size_t compact = (size_t)c->nz * c->hx * c->csz;
    char* a = (char*)c->astage_out[k];
    char* b = a + (size_t)c->nx * c->nz * kIoElem;
    cudaError_t e = cudaSuccess;
    if (c->out_done_rec[k]) e = cudaStreamWaitEvent(s, c->ev_out_done[k], 0);     // the slot's last download is done
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->ko_eta, c->y_eta, compact, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->ko_psi, c->y_psi, compact, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = c->prec == ZK_F32
            ? Pipe<float>::to_physical(c, (cx<float>*)c->ko_eta, (cx<float>*)c->ko_psi, a, b, dtype, s)
            : Pipe<double>::to_physical(c, (cx<double>*)c->ko_eta, (cx<double>*)c->ko_psi, a, b, dtype, s);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_out[k], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->io_out, c->ev_out[k], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(eta, a, n, cudaMemcpyDeviceToHost, c->io_out);
    if (e == cudaSuccess) e = cudaMemcpyAsync(psi, b, n, cudaMemcpyDeviceToHost, c->io_out);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_out_done[k], c->io_out);
    if (e != cudaSuccess) return ZK_ECUDA;
    c->out_done_rec[k] = true;
    return ZK_OK;
}

namespace {
struct CkptHeader {
    char magic[8];
    int version, nx, nz, M, m_run, prec, pad3, has_state, ab_valid, pad_;
    double Lx, Lz, h, g, ab_dt;
};
constexpr char kCkptMagic[8] = {'z', 'k', 'c', 'k', 'p', 't', '0', '1'};
size_t ckpt_compact(const zk_ctx* c) { return (size_t)c->nz * c->hx * c->csz; }
}  // namespace

zk_status zk_checkpoint_size(const zk_ctx* c, size_t* bytes) {
    if (!c || !bytes || c->nb != 1) return ZK_EINVAL;
    *bytes = sizeof(CkptHeader) + 4 * ckpt_compact(c);
    return ZK_OK;
}

zk_status zk_checkpoint_save(zk_ctx* c, void* buf, size_t bytes) {
    size_t need = 0;
    if (!buf || zk_checkpoint_size(c, &need) != ZK_OK || bytes < need) return ZK_EINVAL;
    if (!c->has_state) return ZK_ESTATE;
    CkptHeader hd{};
    std::memcpy(hd.magic, kCkptMagic, sizeof(kCkptMagic));
    hd.version = 1; hd.nx = c->nx; hd.nz = c->nz; hd.M = c->M; hd.m_run = c->m_run; hd.prec = c->prec;
    hd.pad3 = c->pad3 ? 1 : 0; hd.has_state = 1; hd.ab_valid = c->ab_valid ? 1 : 0;
    hd.Lx = c->Lx; hd.Lz = c->Lz; hd.h = c->h; hd.g = c->g; hd.ab_dt = c->ab_dt;
    cudaStream_t s = user_stream(c);
    if (cudaStreamSynchronize(s) != cudaSuccess) return ZK_ECUDA;
    unsigned char* out = static_cast<unsigned char*>(buf);
    std::memcpy(out, &hd, sizeof(hd));
    const size_t n = ckpt_compact(c);
    const void* src[4] = {c->y_eta, c->y_psi, c->h_eta, c->h_psi};
    for (int i = 0; i < 4; ++i)
        if (cudaMemcpy(out + sizeof(hd) + i * n, src[i], n, cudaMemcpyDeviceToHost) != cudaSuccess) return ZK_ECUDA;
    return ZK_OK;
}

zk_status zk_checkpoint_load(zk_ctx* c, const void* buf, size_t bytes) {
    size_t need = 0;
    if (!buf || zk_checkpoint_size(c, &need) != ZK_OK || bytes < need) return ZK_EINVAL;
    CkptHeader hd;
    std::memcpy(&hd, buf, sizeof(hd));
    if (std::memcmp(hd.magic, kCkptMagic, sizeof(kCkptMagic)) != 0 || hd.version != 1 || hd.nx != c->nx ||
        hd.nz != c->nz || hd.M != c->M || hd.prec != c->prec || hd.pad3 != (c->pad3 ? 1 : 0) || hd.Lx != c->Lx ||
        hd.Lz != c->Lz || hd.h != c->h || hd.g != c->g || hd.m_run < 1 || hd.m_run > c->M)
        return ZK_EINVAL;
    if (!hd.has_state) return ZK_ESTATE;
    cudaStream_t s = user_stream(c);
    if (cudaStreamSynchronize(s) != cudaSuccess) return ZK_ECUDA;
    const unsigned char* in = static_cast<const unsigned char*>(buf);
    const size_t n = ckpt_compact(c);
    void* dst[4] = {c->y_eta, c->y_psi, c->h_eta, c->h_psi};
    for (int i = 0; i < 4; ++i)
        if (cudaMemcpy(dst[i], in + sizeof(hd) + i * n, n, cudaMemcpyHostToDevice) != cudaSuccess) return ZK_ECUDA;
    if (hd.m_run != c->m_run) { c->m_run = hd.m_run; drop_graph(c); }
    c->has_state = true;
    c->ab_valid = hd.ab_valid != 0;
    c->ab_dt = hd.ab_dt;
    return ZK_OK;
}

zk_status zk_io_join(zk_ctx* c) {
    if (!c) return ZK_EINVAL;
    if (!c->io) return ZK_OK;
    cudaError_t r = cudaSuccess;
    for (cudaStream_t q : {c->io, c->io_out}) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return ZK_ECUDA;
        r = cudaEventRecord(e, q);
        if (r == cudaSuccess) r = cudaStreamWaitEvent(user_stream(c), e, 0);
        cudaEventDestroy(e);
        if (r != cudaSuccess) break;
    }
    return cu(r);
}

zk_status zk_device_bytes(const zk_ctx* c, size_t* b) {
    if (!c || !b) return ZK_EINVAL;
    *b = c->bytes;
    return ZK_OK;
}

zk_status zk_launches_per_step(const zk_ctx* c, int* n) {
    if (!c || !n) return ZK_EINVAL;
    *n = c->gvalid ? c->launches_per_step : (c->opt.integrator == ZK_IFAB2 ? 1 : 4) * (2 * c->M + 1);
    return ZK_OK;
}

static zk_status closure_buffers(zk_ctx* c) {
    if (c->cspec) return ZK_OK;
    const size_t compact = (size_t)c->nz * c->hx * c->csz, plane = (size_t)c->nx * c->nz * sizeof(float);
    zk_status st = dalloc(c, &c->cspec, 6 * compact);
    if (st == ZK_OK) st = dalloc(c, &c->feat, 6 * plane);
    if (st == ZK_OK && !c->chk) st = dalloc(c, &c->chk, 2 * compact);
    if (st == ZK_OK && !c->cpart) st = dalloc(c, (void**)&c->cpart, 2 * 256 * sizeof(double));
    return st;
}

static void set_scales(zk_ctx* c, const float* in_scale, const float* out_scale) {
    for (int i = 0; i < 6; ++i) c->sc.in[i] = in_scale ? in_scale[i] : 1.0f;
    for (int i = 0; i < 2; ++i) c->sc.out[i] = out_scale ? out_scale[i] : 1.0f;
}

static bool scales_ok(const float* in_scale, const float* out_scale) {
    for (int i = 0; in_scale && i < 6; ++i) if (!(in_scale[i] > 0.0f) || !std::isfinite(in_scale[i])) return false;
    for (int i = 0; out_scale && i < 2; ++i) if (!(out_scale[i] > 0.0f) || !std::isfinite(out_scale[i])) return false;
    return true;
}

zk_status zk_closure_features(zk_ctx* c, int base_order, const float* in_scale, const float* out_scale, float* feat,
                              float* target) {
    if (!c || !feat || base_order < 1 || base_order >= c->M || !scales_ok(in_scale, out_scale)) return ZK_EINVAL;
    if (c->prec != ZK_F32) return ZK_EUNSUPPORTED;
    if (!c->has_state) return ZK_ESTATE;
    zk_status st = closure_buffers(c);
    if (st != ZK_OK) return st;
    const ClosureScales keep = c->sc;
    const int keep_base = c->base_M;
    set_scales(c, in_scale, out_scale);
    c->base_M = base_order;
    cudaStream_t s = user_stream(c);
    cudaError_t e = Pipe<float>::closure_features(c, feat, target, s);
    c->sc = keep;
    c->base_M = keep_base;
    if (e != cudaSuccess) return ZK_ECUDA;
    return cu(cudaStreamSynchronize(s));
}

zk_status zk_closure_set(zk_ctx* c, zk_net* net, int base_order, const float* in_scale, const float* out_scale,
                         int check_every, double check_tol) {
    if (!c) return ZK_EINVAL;
    if (!net) {
        c->closure_on = false;
        c->net = nullptr;
        drop_graph(c);
        return ZK_OK;
    }
    if (base_order < 1 || base_order >= c->M || check_every < 0 || !(check_tol > 0) || !in_scale || !out_scale ||
        !scales_ok(in_scale, out_scale))
        return ZK_EINVAL;
    if (c->prec != ZK_F32 || c->adapt_every > 0) return ZK_EUNSUPPORTED;
    zk_status st = closure_buffers(c);
    if (st == ZK_OK) st = zk_net_reserve(net, (size_t)c->nx * c->nz);
    if (st != ZK_OK) return st;
    c->net = net;
    c->base_M = base_order;
    set_scales(c, in_scale, out_scale);
    c->check_every = check_every;
    c->check_tol = check_tol;
    c->closure_on = true;
    c->nchecks = 0;
    c->nsteps = 0;
    c->fallback_step = -1;
    c->last_err = -1.0;
    drop_graph(c);
    return ZK_OK;
}

zk_status zk_closure_set_once_per_step(zk_ctx* c, int on) {
    if (!c || (on != 0 && on != 1)) return ZK_EINVAL;
    if (c->closure_once != (on == 1)) {
        c->closure_once = on == 1;
        drop_graph(c);
    }
    return ZK_OK;
}

zk_status zk_set_series_fp64(zk_ctx* c, int on) {
    if (!c || (on != 0 && on != 1)) return ZK_EINVAL;
    if (c->prec != ZK_F32) return ZK_OK;   // FP64 contexts sum in FP64 already
    if ((c->pad3 || c->dft_split != ZK_DFT_F32) && on) return ZK_EUNSUPPORTED;
    if (c->series64 != (on == 1)) {
        c->series64 = on == 1;
        drop_graph(c);
    }
    return ZK_OK;
}

zk_status zk_set_dft_precision(zk_ctx* c, int mode) {
    if (!c || mode < ZK_DFT_F32 || mode > ZK_DFT_FP16X3) return ZK_EINVAL;
    if (mode != ZK_DFT_F32) {
        auto long_line = [](int n) { return n == 1536 || n == 3072; };
        if (c->prec != ZK_F32 || c->pad3 || c->series64 || c->nb > 1 || !long_line(c->npx) || !long_line(c->npz))
            return ZK_EUNSUPPORTED;
    }
    if (c->dft_split != mode) {
        c->dft_split = mode;
        // the split plans keep the radices, and so the twiddle tables, of the default plan
        const int v = mode != ZK_DFT_F32 ? 0 : c->plan_v;
        c->tw_px = c->tw_pv[v][0];
        c->tw_pz = c->tw_pv[v][1];
        drop_graph(c);
    }
    return ZK_OK;
}

zk_status zk_set_adaptive_order(zk_ctx* c, int m_min, double tol, int check_every) {
    if (!c || check_every < 0) return ZK_EINVAL;
    if (check_every == 0) {
        c->adapt_every = 0;
        if (c->m_run != c->M) { c->m_run = c->M; drop_graph(c); }
        return ZK_OK;
    }
    if (m_min < 1 || m_min > c->M || !(tol >= 0.0) || !std::isfinite(tol)) return ZK_EINVAL;
    if (c->closure_on) return ZK_EUNSUPPORTED;
    zk_status st = ZK_OK;
    if (!c->chk) st = dalloc(c, &c->chk, 2 * (size_t)c->nz * c->hx * c->csz);
    if (st == ZK_OK && !c->cpart) st = dalloc(c, (void**)&c->cpart, 2 * 256 * sizeof(double));
    if (st != ZK_OK) return st;
    c->adapt_every = check_every;
    c->adapt_min = m_min;
    c->adapt_tol = tol;
    c->adapt_checks = 0;
    c->nsteps = 0;
    return ZK_OK;
}

zk_status zk_adaptive_status(const zk_ctx* c, int* order, int* checks, double* err) {
    if (!c) return ZK_EINVAL;
    if (order) *order = c->m_run > 0 ? c->m_run : c->M;
    if (checks) *checks = c->adapt_checks;
    if (err) for (int m = 1; m <= ZK_MAX_ORDER; ++m) err[m - 1] = c->adapt_err[m];
    return ZK_OK;
}

zk_status zk_closure_status(const zk_ctx* c, int* active, int* checks, long long* fallback_step, double* last_err) {
    if (!c) return ZK_EINVAL;
    if (active) *active = c->closure_on ? 1 : 0;
    if (checks) *checks = c->nchecks;
    if (fallback_step) *fallback_step = c->fallback_step;
    if (last_err) *last_err = c->last_err;
    return ZK_OK;
}

}  // extern "C"

// ===========================================================================
// Batched tiles: groups of tiles that share grid and order, one launch per
// pass of a group (blockIdx.y = tile), the groups as parallel branches of one
// captured step graph.
// ===========================================================================
struct zk_batch {
    int ntiles = 0, prec = ZK_F32;
    std::vector<zk_ctx*> groups;
    std::vector<std::pair<int, int>> where;    // tile -> (group, index in group)
    std::vector<char> has_state;
    std::vector<cudaStream_t> gs;              // one capture branch per group
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaStream_t cap = nullptr;
    zk_options opt{};
    cudaGraphExec_t gexec = nullptr, gexec_boot = nullptr;
    bool gvalid = false;
    double gdt = 0.0;
    bool ab_valid = false;
    double ab_dt = 0.0;
    int launches_per_step = 0;
};

namespace {

void batch_drop_graph(zk_batch* b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->gexec_boot) cudaGraphExecDestroy(b->gexec_boot);
    b->gexec = b->gexec_boot = nullptr;
    b->gvalid = false;
}

zk_status batch_capture(zk_batch* b, double dt, int variant, cudaGraphExec_t* out, int* nl) {
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) return ZK_ECUDA;
    cudaError_t e = cudaEventRecord(b->fork, b->cap);
    // every forked branch is joined back, also after a failed enqueue, so
    // that the capture ends with no stream left capturing
    for (size_t i = 0; i < b->groups.size() && e == cudaSuccess; ++i) {
        e = cudaStreamWaitEvent(b->gs[i], b->fork, 0);
        if (e != cudaSuccess) break;
        const cudaError_t eq = enqueue_step_any(b->groups[i], dt, b->gs[i], nl, variant);
        e = cudaEventRecord(b->join[i], b->gs[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->join[i], 0);
        if (e == cudaSuccess) e = eq;
    }
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return ZK_ECUDA;
    }
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { *out = nullptr; return ZK_ECUDA; }
    return ZK_OK;
}

zk_status batch_build_graph(zk_batch* b, double dt) {
    batch_drop_graph(b);
    int nl = 0;
    zk_status st;
    if (b->opt.integrator == ZK_IFAB2) {
        st = batch_capture(b, dt, 1, &b->gexec_boot, &nl);
        nl = 0;
        if (st == ZK_OK) st = batch_capture(b, dt, 2, &b->gexec, &nl);
    } else {
        st = batch_capture(b, dt, 0, &b->gexec, &nl);
    }
    if (st != ZK_OK) { batch_drop_graph(b); return st; }
    b->gvalid = true;
    b->gdt = dt;
    b->launches_per_step = nl;
    return ZK_OK;
}

// Tuning cache: a JSON object {"entries": {"<key>": {"plan_v": v, "col_ci": c,
// "row_occ": o, "ms": t}, ...}} with one entry per line; the key names the
// device, grid, order, precision and tile count.
std::string tune_key(const zk_ctx* c) {
    cudaDeviceProp pr;
    std::string dev = "gpu";
    if (cudaGetDeviceProperties(&pr, c->device) == cudaSuccess) dev = pr.name;
    for (char& ch : dev) if (ch == '"' || ch == '\\') ch = '_';
    char k[256];
    snprintf(k, sizeof(k), "%s/%dx%d/M%d/%s/nb%d", dev.c_str(), c->nx, c->nz, c->M, c->prec == ZK_F32 ? "f32" : "f64", c->nb);
    return k;
}

struct TuneEntry { int plan_v, col_ci, row_occ; double ms; };

std::vector<std::pair<std::string, TuneEntry>> tune_load(const char* path) {
    std::vector<std::pair<std::string, TuneEntry>> out;
    if (!path) return out;
    FILE* f = fopen(path, "r");
    if (!f) return out;
    char line[1024];
    while (fgets(line, sizeof(line), f)) {
        const char* q0 = strchr(line, '"');
        if (!q0) continue;
        const char* q1 = strchr(q0 + 1, '"');
        if (!q1) continue;
        const char* body = strstr(q1, "\"plan_v\"");
        if (!body) continue;
        TuneEntry t{};
        if (sscanf(body, "\"plan_v\": %d, \"col_ci\": %d, \"row_occ\": %d, \"ms\": %lf", &t.plan_v, &t.col_ci,
                   &t.row_occ, &t.ms) == 4 &&
            t.plan_v >= 0 && t.plan_v <= 1 && t.col_ci >= 0 && t.col_ci <= 2 && t.row_occ >= 0 && t.row_occ <= 64)
            out.push_back({std::string(q0 + 1, q1), t});
    }
    fclose(f);
    return out;
}

bool tune_save(const char* path, const std::vector<std::pair<std::string, TuneEntry>>& es) {
    if (!path) return true;
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return false;
    fprintf(f, "{\"version\": 1, \"entries\": {\n");
    for (size_t i = 0; i < es.size(); ++i)
        fprintf(f, "\"%s\": {\"plan_v\": %d, \"col_ci\": %d, \"row_occ\": %d, \"ms\": %.6f}%s\n", es[i].first.c_str(),
                es[i].second.plan_v, es[i].second.col_ci, es[i].second.row_occ, es[i].second.ms,
                i + 1 < es.size() ? "," : "");
    fprintf(f, "}}\n");
    const bool ok = fclose(f) == 0;
    return ok && rename(tmp.c_str(), path) == 0;
}

// Mean ms of one eager step of group c under the launch shape (v, ci, occ), or
// a negative value when the shape cannot launch (threads or shared memory).
double time_shape(zk_ctx* c, double dt, int v, int ci, int occ, cudaStream_t s, int reps) {
    c->plan_v = v; c->col_ci = ci; c->row_occ = occ;
    c->tw_px = c->tw_pv[v][0];
    c->tw_pz = c->tw_pv[v][1];
    const int variant = c->opt.integrator == ZK_IFAB2 ? 1 : 0;
    if (enqueue_step_any(c, dt, s, nullptr, variant) != cudaSuccess) { cudaStreamSynchronize(s); cudaGetLastError(); return -1.0; }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = enqueue_step_any(c, dt, s, nullptr, variant);
    cudaEventRecord(e1, s);
    cudaError_t es = cudaStreamSynchronize(s);
    float ms = -1.f;
    if (e == cudaSuccess && es == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    return (e == cudaSuccess && es == cudaSuccess) ? ms / reps : -1.0;
}

}  // namespace

extern "C" {

void zk_batch_destroy(zk_batch* b) {
    if (!b) return;
    batch_drop_graph(b);
    for (zk_ctx* c : b->groups) zk_destroy(c);
    for (cudaStream_t s : b->gs) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->join) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

zk_status zk_batch_create(zk_batch** out, int ntiles, const int* nx, const int* nz, const double* Lx,
                          const double* Lz, const double* h, double g, const int* M, int precision) {
    if (!out || ntiles < 1 || !nx || !nz || !Lx || !Lz || !h || !M) return ZK_EINVAL;
    *out = nullptr;
    zk_batch* b = new (std::nothrow) zk_batch();
    if (!b) return ZK_ENOMEM;
    b->ntiles = ntiles;
    b->prec = precision;
    b->where.resize(ntiles);
    b->has_state.assign(ntiles, 0);
    // group tiles by (nx, nz, Lx, Lz, M) in order of first appearance
    std::vector<std::vector<int>> members;
    for (int t = 0; t < ntiles; ++t) {
        int gi = -1;
        for (size_t k = 0; k < members.size(); ++k) {
            const int r = members[k][0];
            if (nx[r] == nx[t] && nz[r] == nz[t] && Lx[r] == Lx[t] && Lz[r] == Lz[t] && M[r] == M[t]) { gi = (int)k; break; }
        }
        if (gi < 0) { gi = (int)members.size(); members.emplace_back(); }
        b->where[t] = {gi, (int)members[gi].size()};
        members[gi].push_back(t);
    }
    zk_status st = ZK_OK;
    for (size_t k = 0; k < members.size() && st == ZK_OK; ++k) {
        const int r = members[k][0];
        std::vector<double> hs;
        for (int t : members[k]) hs.push_back(h[t]);
        zk_ctx* c = nullptr;
        st = ctx_create(&c, nx[r], nz[r], Lx[r], Lz[r], hs.data(), (int)hs.size(), g, M[r], precision);
        if (st == ZK_OK) {
            b->groups.push_back(c);
            cudaStream_t s = nullptr;
            cudaEvent_t e = nullptr;
            if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) st = ZK_ECUDA;
            else b->gs.push_back(s);
            if (st == ZK_OK && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) st = ZK_ECUDA;
            else if (st == ZK_OK) b->join.push_back(e);
        }
    }
    if (st == ZK_OK && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) st = ZK_ECUDA;
    if (st == ZK_OK && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) st = ZK_ECUDA;
    b->opt.eps = 1.0; b->opt.integrator = ZK_RK4; b->opt.taper = 1; b->opt.filter = 1; b->opt.stream = nullptr;
    if (st != ZK_OK) { zk_batch_destroy(b); return st; }
    *out = b;
    return ZK_OK;
}

zk_status zk_batch_set_options(zk_batch* b, const zk_options* o) {
    if (!b || !o) return ZK_EINVAL;
    for (zk_ctx* c : b->groups) {
        zk_status st = zk_set_options(c, o);
        if (st != ZK_OK) return st;
    }
    if (o->integrator != b->opt.integrator || o->eps != b->opt.eps || o->taper != b->opt.taper) b->ab_valid = false;
    b->opt = *o;
    batch_drop_graph(b);
    return ZK_OK;
}

zk_status zk_batch_set_state(zk_batch* b, int tile, const void* eta, const void* psi, int dtype, int on_device) {
    if (!b || tile < 0 || tile >= b->ntiles) return ZK_EINVAL;
    zk_ctx v;
    tile_view(b->groups[b->where[tile].first], b->where[tile].second, &v);
    zk_status st = zk_set_state(&v, eta, psi, dtype, on_device);
    if (st == ZK_OK) { b->has_state[tile] = 1; b->ab_valid = false; }
    return st;
}

zk_status zk_batch_get_state(zk_batch* b, int tile, void* eta, void* psi, int dtype, int on_device) {
    if (!b || tile < 0 || tile >= b->ntiles) return ZK_EINVAL;
    if (!b->has_state[tile]) return ZK_ESTATE;
    zk_ctx v;
    tile_view(b->groups[b->where[tile].first], b->where[tile].second, &v);
    return zk_get_state(&v, eta, psi, dtype, on_device);
}

zk_status zk_batch_energy(zk_batch* b, int tile, double* H, double* kin, double* pot, double* mean_eta) {
    if (!b || tile < 0 || tile >= b->ntiles) return ZK_EINVAL;
    if (!b->has_state[tile]) return ZK_ESTATE;
    zk_ctx v;
    tile_view(b->groups[b->where[tile].first], b->where[tile].second, &v);
    return zk_energy(&v, H, kin, pot, mean_eta);
}

zk_status zk_batch_step(zk_batch* b, double dt, int n) {
    if (!b || n < 0 || !(dt > 0) || !std::isfinite(dt)) return ZK_EINVAL;
    for (int t = 0; t < b->ntiles; ++t) if (!b->has_state[t]) return ZK_ESTATE;
    if (n == 0) return ZK_OK;
    if (!b->gvalid || b->gdt != dt) {
        zk_status st = batch_build_graph(b, dt);
        if (st != ZK_OK) return st;
    }
    cudaStream_t s = (cudaStream_t)b->opt.stream;
    for (int i = 0; i < n; ++i) {
        cudaGraphExec_t g = b->gexec;
        if (b->opt.integrator == ZK_IFAB2 && !(b->ab_valid && b->ab_dt == dt)) {
            g = b->gexec_boot;
            b->ab_valid = true;
            b->ab_dt = dt;
        }
        if (cudaGraphLaunch(g, s) != cudaSuccess) return ZK_ECUDA;
    }
    return ZK_OK;
}

zk_status zk_batch_sync(zk_batch* b) {
    if (!b) return ZK_EINVAL;
    return cu(cudaStreamSynchronize((cudaStream_t)b->opt.stream));
}

zk_status zk_batch_info(const zk_batch* b, int* ngroups, int* launches_per_step, size_t* device_bytes) {
    if (!b) return ZK_EINVAL;
    if (ngroups) *ngroups = (int)b->groups.size();
    if (launches_per_step) {
        int n = 0;
        for (const zk_ctx* c : b->groups) n += (b->opt.integrator == ZK_IFAB2 ? 1 : 4) * (2 * c->M + 1);
        *launches_per_step = n;
    }
    if (device_bytes) {
        size_t by = 0;
        for (const zk_ctx* c : b->groups) by += c->bytes;
        *device_bytes = by;
    }
    return ZK_OK;
}

zk_status zk_batch_group(const zk_batch* b, int gi, int* nx, int* nz, int* M, int* ntiles, int* plan_v, int* col_ci,
                         int* row_occ) {
    if (!b || gi < 0 || gi >= (int)b->groups.size()) return ZK_EINVAL;
    const zk_ctx* c = b->groups[gi];
    if (nx) *nx = c->nx;
    if (nz) *nz = c->nz;
    if (M) *M = c->M;
    if (ntiles) *ntiles = c->nb;
    if (plan_v) *plan_v = c->plan_v;
    if (col_ci) *col_ci = c->col_ci;
    if (row_occ) *row_occ = c->row_occ;
    return ZK_OK;
}

zk_status zk_batch_set_shape(zk_batch* b, int gi, int plan_v, int col_ci, int row_occ) {
    if (!b || gi < 0 || gi >= (int)b->groups.size()) return ZK_EINVAL;
    if (plan_v < 0 || plan_v > 1 || col_ci < 0 || col_ci > 2 || row_occ < 0 || row_occ > 64) return ZK_EINVAL;
    zk_ctx* c = b->groups[gi];
    c->plan_v = plan_v; c->col_ci = col_ci; c->row_occ = row_occ;
    c->tw_px = c->tw_pv[plan_v][0];
    c->tw_pz = c->tw_pv[plan_v][1];
    batch_drop_graph(b);
    return ZK_OK;
}

zk_status zk_batch_autotune(zk_batch* b, double dt, const char* cache_path, int* tuned, int* cached) {
    if (!b || !(dt > 0) || !std::isfinite(dt)) return ZK_EINVAL;
    for (int t = 0; t < b->ntiles; ++t) if (!b->has_state[t]) return ZK_ESTATE;
    if (cudaStreamSynchronize((cudaStream_t)b->opt.stream) != cudaSuccess) return ZK_ECUDA;   // states set
    auto cache = tune_load(cache_path);
    int nt = 0, nc = 0;
    bool dirty = false;
    zk_status st = ZK_OK;
    for (size_t gi = 0; gi < b->groups.size() && st == ZK_OK; ++gi) {
        zk_ctx* c = b->groups[gi];
        const std::string key = tune_key(c);
        const TuneEntry* hit = nullptr;
        for (auto& kv : cache) if (kv.first == key) hit = &kv.second;
        if (hit) {
            zk_batch_set_shape(b, (int)gi, hit->plan_v, hit->col_ci, hit->row_occ);
            ++nc;
            continue;
        }
        // the timing steps advance the group: keep its state and forcing history
        cudaStream_t s = b->gs[gi];
        const size_t bytes = (size_t)c->tst * c->csz * c->nb;
        void* save = nullptr;
        if (cudaMalloc(&save, 4 * bytes) != cudaSuccess) { cudaGetLastError(); return ZK_ENOMEM; }
        void* src[4] = {c->y_eta, c->y_psi, c->h_eta, c->h_psi};
        for (int i = 0; i < 4; ++i) cudaMemcpyAsync((char*)save + i * bytes, src[i], bytes, cudaMemcpyDeviceToDevice, s);
        const bool var = plan_has_variant(c->npx) || plan_has_variant(c->npz);
        TuneEntry best{0, 1, 0, -1.0};
        for (int v = 0; v <= (var && c->prec == ZK_F32 ? 1 : 0); ++v)
            for (int ci = 0; ci <= 2; ++ci)
                for (int occ : {0, 1, 2}) {
                    if (c->prec != ZK_F32 && ci != 1) continue;
                    const double ms = time_shape(c, dt, v, ci, occ, s, 3);
                    if (ms > 0 && (best.ms < 0 || ms < best.ms)) best = {v, ci, occ, ms};
                }
        for (int i = 0; i < 4; ++i) cudaMemcpyAsync(src[i], (char*)save + i * bytes, bytes, cudaMemcpyDeviceToDevice, s);
        cudaError_t e = cudaStreamSynchronize(s);
        cudaFree(save);
        if (e != cudaSuccess) return ZK_ECUDA;
        if (best.ms < 0) { best = {0, 1, 0, 0.0}; st = ZK_ECUDA; }
        zk_batch_set_shape(b, (int)gi, best.plan_v, best.col_ci, best.row_occ);
        cache.push_back({key, best});
        dirty = true;
        ++nt;
    }
    b->ab_valid = false;   // the timing steps used the history buffers
    if (dirty && !tune_save(cache_path, cache) && st == ZK_OK) st = ZK_EINVAL;
    if (tuned) *tuned = nt;
    if (cached) *cached = nc;
    return st;
}

}  // extern "C"
