// zk_launch_impl.cuh - the launch functions of the row and column kernels, dispatched on
// the compile-time padded line lengths, plan variants, precision and padding. Included
// only by the zk_launch_{row,col}_{f32,f64}.cu units, each of which instantiates one.
#pragma once

#include <algorithm>

#include "zk_launch.h"

namespace zk {

template <typename T, int NPX, int V, typename TA = T, int DIV = 3>
cudaError_t launch_row_t(const RowArgs<T>& a, const cx<T>* tw, int npz, cudaStream_t s) {
    constexpr int TL = IPlan<NPX, V>::TL;
    // narrow groups: one line per group, rounded to whole warps; wide groups:
    // at most 1024 threads, lines beyond that taken in waves
    int nl = a.nlines, groups;
    if constexpr (TL < 32) { constexpr int per = 32 / TL; nl = (nl + per - 1) / per * per; groups = nl; }
    else groups = std::min(nl, std::max(1, kRowMaxThreads / TL));
    const int threads = groups * TL;
    const size_t smem = (size_t)nl * line_stride(NPX) * sizeof(cx<T>);
    if (threads > 1024 || smem > (size_t)smem_optin()) return cudaErrorInvalidConfiguration;
    // a block of one wide line group synchronises on barrier 0 alone (more blocks per SM)
    const bool oneg = TL >= 32 && groups == 1;
    const void* fn = oneg ? (const void*)row2_kernel<T, NPX, V, TA, DIV, true>
                          : (const void*)row2_kernel<T, NPX, V, TA, DIV, false>;
    cudaError_t e = ensure_smem(fn, smem);
    if (e != cudaSuccess) return e;
    RowArgs<T> b = a;
    b.npz = npz;
    // persistent over rows: the resident blocks (capped at a.occ per SM when
    // set) shared among the a.nb tiles of the launch
    int per_sm = 1, sms = 1;
    occupancy(fn, threads, smem, &per_sm, &sms);
    if (a.occ > 0) per_sm = std::min(per_sm, a.occ);
    const int nb = std::max(1, a.nb);
    const int gx = std::max(1, std::min(npz, (per_sm * sms + nb - 1) / nb));
    if (oneg) row2_kernel<T, NPX, V, TA, DIV, true><<<dim3(gx, nb), threads, smem, s>>>(b, tw);
    else row2_kernel<T, NPX, V, TA, DIV, false><<<dim3(gx, nb), threads, smem, s>>>(b, tw);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_row(int npx, int v, const RowArgs<T>& a, const cx<T>* tw, int npz, cudaStream_t s) {
    if (v == SPLIT_BF16 || v == SPLIT_FP16) {   // FP32 3/2-rule plans of the long lines only
        if constexpr (sizeof(T) == 4) {
            if (a.pad3 || a.acc64) return cudaErrorInvalidValue;
            switch (npx * 4 + v) {
            case 1536 * 4 + SPLIT_BF16: return launch_row_t<T, 1536, SPLIT_BF16>(a, tw, npz, s);
            case 3072 * 4 + SPLIT_BF16: return launch_row_t<T, 3072, SPLIT_BF16>(a, tw, npz, s);
            case 1536 * 4 + SPLIT_FP16: return launch_row_t<T, 1536, SPLIT_FP16>(a, tw, npz, s);
            case 3072 * 4 + SPLIT_FP16: return launch_row_t<T, 3072, SPLIT_FP16>(a, tw, npz, s);
            default: break;
            }
        }
        return cudaErrorInvalidValue;
    }
    if constexpr (sizeof(T) == 4) {
        if (a.pad3) {    // 3N padding: FP32, default plans and sums
            switch (npx) {
            case 48: return launch_row_t<T, 48, 0, T, 6>(a, tw, npz, s);
            case 96: return launch_row_t<T, 96, 0, T, 6>(a, tw, npz, s);
            case 192: return launch_row_t<T, 192, 0, T, 6>(a, tw, npz, s);
            case 384: return launch_row_t<T, 384, 0, T, 6>(a, tw, npz, s);
            case 768: return launch_row_t<T, 768, 0, T, 6>(a, tw, npz, s);
            case 1536: return launch_row_t<T, 1536, 0, T, 6>(a, tw, npz, s);
            case 3072: return launch_row_t<T, 3072, 0, T, 6>(a, tw, npz, s);
            default: return cudaErrorInvalidValue;
            }
        }
        if (a.acc64) {   // FP64 series sums: default plans only
            switch (npx) {
            case 24: return launch_row_t<T, 24, 0, double>(a, tw, npz, s);
            case 48: return launch_row_t<T, 48, 0, double>(a, tw, npz, s);
            case 96: return launch_row_t<T, 96, 0, double>(a, tw, npz, s);
            case 192: return launch_row_t<T, 192, 0, double>(a, tw, npz, s);
            case 384: return launch_row_t<T, 384, 0, double>(a, tw, npz, s);
            case 768: return launch_row_t<T, 768, 0, double>(a, tw, npz, s);
            case 1536: return launch_row_t<T, 1536, 0, double>(a, tw, npz, s);
            case 3072: return launch_row_t<T, 3072, 0, double>(a, tw, npz, s);
            default: return cudaErrorInvalidValue;
            }
        }
        if (v == 1) {
            switch (npx) {
            case 768: return launch_row_t<T, 768, 1>(a, tw, npz, s);
            case 1536: return launch_row_t<T, 1536, 1>(a, tw, npz, s);
            case 3072: return launch_row_t<T, 3072, 1>(a, tw, npz, s);
            default: break;
            }
        }
    }
    switch (npx) {
    case 24: return launch_row_t<T, 24, 0>(a, tw, npz, s);
    case 48: return launch_row_t<T, 48, 0>(a, tw, npz, s);
    case 96: return launch_row_t<T, 96, 0>(a, tw, npz, s);
    case 192: return launch_row_t<T, 192, 0>(a, tw, npz, s);
    case 384: return launch_row_t<T, 384, 0>(a, tw, npz, s);
    case 768: return launch_row_t<T, 768, 0>(a, tw, npz, s);
    case 1536: return launch_row_t<T, 1536, 0>(a, tw, npz, s);
    case 3072: if constexpr (sizeof(T) == 4) return launch_row_t<T, 3072, 0>(a, tw, npz, s); else return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
}

template <typename T, int NPZ, int CB, int V, int DIV = 3>
cudaError_t launch_col_t(const ColArgs<T>& a, const cx<T>* tw, cudaStream_t s, int* nblocks) {
    constexpr int TL = IPlan<NPZ, V>::TL;
    const int threads = CB * TL < 32 ? 32 : CB * TL;
    const int groups = threads / TL;
    const size_t smem = col_smem_bytes<T, NPZ, DIV>(a.kind == COL_FINAL, groups);
    if (threads > 1024 || smem > (size_t)smem_optin()) return cudaErrorInvalidConfiguration;
    const int grid = (a.hx + CB - 1) / CB;
    if (nblocks) *nblocks = grid;
    cudaError_t e = ensure_smem((const void*)col2_kernel<T, NPZ, CB, V, DIV>, smem);
    if (e != cudaSuccess) return e;
    col2_kernel<T, NPZ, CB, V, DIV><<<dim3(grid, std::max(1, a.nb)), threads, smem, s>>>(a, tw);
    return cudaGetLastError();
}

// Columns-per-block choice ci (0 / 1 / 2 = half / default / double) is tuned
// for FP32 lines of 192 and longer; everything else runs the default.
template <typename T, int NPZ, int V>
cudaError_t launch_col_v(int ci, const ColArgs<T>& a, const cx<T>* tw, cudaStream_t s, int* nblocks) {
    constexpr int ES = (int)sizeof(cx<T>);
    if constexpr (ES == 8 && NPZ >= 192) {
        if (ci == 0) return launch_col_t<T, NPZ, col_cb_pick<NPZ, ES, V>(0), V>(a, tw, s, nblocks);
        if (ci == 2) return launch_col_t<T, NPZ, col_cb_pick<NPZ, ES, V>(2), V>(a, tw, s, nblocks);
    }
    return launch_col_t<T, NPZ, col_cb<NPZ, ES, V>(), V>(a, tw, s, nblocks);
}

template <typename T>
cudaError_t launch_col(int npz, int v, int ci, const ColArgs<T>& a, const cx<T>* tw, cudaStream_t s,
                       int* nblocks) {
    if (v == SPLIT_BF16 || v == SPLIT_FP16) {   // default blocking; FP32 3/2-rule plans of the long lines
        if constexpr (sizeof(T) == 4) {
            constexpr int ES = (int)sizeof(cx<T>);
            if (a.pad3) return cudaErrorInvalidValue;
            switch (npz * 4 + v) {
            case 1536 * 4 + SPLIT_BF16:
                return launch_col_t<T, 1536, col_cb<1536, ES, SPLIT_BF16>(), SPLIT_BF16>(a, tw, s, nblocks);
            case 3072 * 4 + SPLIT_BF16:
                return launch_col_t<T, 3072, col_cb<3072, ES, SPLIT_BF16>(), SPLIT_BF16>(a, tw, s, nblocks);
            case 1536 * 4 + SPLIT_FP16:
                return launch_col_t<T, 1536, col_cb<1536, ES, SPLIT_FP16>(), SPLIT_FP16>(a, tw, s, nblocks);
            case 3072 * 4 + SPLIT_FP16:
                return launch_col_t<T, 3072, col_cb<3072, ES, SPLIT_FP16>(), SPLIT_FP16>(a, tw, s, nblocks);
            default: break;
            }
        }
        return cudaErrorInvalidValue;
    }
    if constexpr (sizeof(T) == 4) {
        if (a.pad3) {    // 3N padding: FP32, default plans and blocking
            constexpr int ES = (int)sizeof(cx<T>);
            switch (npz) {
            case 48: return launch_col_t<T, 48, col_cb<48, ES>(), 0, 6>(a, tw, s, nblocks);
            case 96: return launch_col_t<T, 96, col_cb<96, ES>(), 0, 6>(a, tw, s, nblocks);
            case 192: return launch_col_t<T, 192, col_cb<192, ES>(), 0, 6>(a, tw, s, nblocks);
            case 384: return launch_col_t<T, 384, col_cb<384, ES>(), 0, 6>(a, tw, s, nblocks);
            case 768: return launch_col_t<T, 768, col_cb<768, ES>(), 0, 6>(a, tw, s, nblocks);
            case 1536: return launch_col_t<T, 1536, col_cb<1536, ES>(), 0, 6>(a, tw, s, nblocks);
            case 3072: return launch_col_t<T, 3072, col_cb<3072, ES>(), 0, 6>(a, tw, s, nblocks);
            default: return cudaErrorInvalidValue;
            }
        }
        if (v == 1) {
            switch (npz) {
            case 768: return launch_col_v<T, 768, 1>(ci, a, tw, s, nblocks);
            case 1536: return launch_col_v<T, 1536, 1>(ci, a, tw, s, nblocks);
            case 3072: return launch_col_v<T, 3072, 1>(ci, a, tw, s, nblocks);
            default: break;
            }
        }
    }
    switch (npz) {
    case 24: return launch_col_v<T, 24, 0>(ci, a, tw, s, nblocks);
    case 48: return launch_col_v<T, 48, 0>(ci, a, tw, s, nblocks);
    case 96: return launch_col_v<T, 96, 0>(ci, a, tw, s, nblocks);
    case 192: return launch_col_v<T, 192, 0>(ci, a, tw, s, nblocks);
    case 384: return launch_col_v<T, 384, 0>(ci, a, tw, s, nblocks);
    case 768: return launch_col_v<T, 768, 0>(ci, a, tw, s, nblocks);
    case 1536: return launch_col_v<T, 1536, 0>(ci, a, tw, s, nblocks);
    case 3072: if constexpr (sizeof(T) == 4) return launch_col_v<T, 3072, 0>(ci, a, tw, s, nblocks); else return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace zk
