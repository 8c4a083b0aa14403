// zk_launch_common.cu - occupancy and shared-memory helpers shared by the launch units.
#include <algorithm>
#include <cstdio>
#include <mutex>
#include <string>
#include <unordered_map>

#include "zk_launch.h"

namespace zk {

namespace {
std::mutex g_occ_mu;
std::unordered_map<std::string, std::pair<int, int>> g_occ;
std::mutex g_attr_mu;
std::unordered_map<const void*, int> g_attr;
}  // namespace

void occupancy(const void* fn, int threads, size_t smem, int* per_sm, int* sms) {
    char key[96];
    snprintf(key, sizeof(key), "%p/%d/%zu", fn, threads, smem);
    {
        std::lock_guard<std::mutex> lk(g_occ_mu);
        auto it = g_occ.find(key);
        if (it != g_occ.end()) { *per_sm = it->second.first; *sms = it->second.second; return; }
    }
    int dev = 0, n = 0, nb = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem);
    *per_sm = std::max(1, nb);
    *sms = std::max(1, n);
    std::lock_guard<std::mutex> lk(g_occ_mu);
    g_occ[key] = {*per_sm, *sms};
}

int smem_optin() {
    static int v = -1;
    if (v < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    }
    return v;
}

cudaError_t ensure_smem(const void* fn, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    std::lock_guard<std::mutex> lk(g_attr_mu);
    auto it = g_attr.find(fn);
    if (it != g_attr.end() && it->second >= (int)bytes) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) g_attr[fn] = (int)bytes;
    return e;
}

}  // namespace zk
