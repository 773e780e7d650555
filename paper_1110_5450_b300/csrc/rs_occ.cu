// rs_occ.cu -- resident CTAs per SM, answered from a per-kernel table.
//
// Plans and server launches size their grids from the runtime's occupancy
// query, and the streaming set-up asks it for every candidate strip width.
// Occupancy falls in steps as a CTA's dynamic shared memory grows, so the
// first request for a (device, kernel, block size) finds each step by
// bisection and every later one is a table lookup with no CUDA call.
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "rs_internal.h"

namespace rs {

namespace {

constexpr size_t kSmemMax = 227 * 1024;

struct OccTable {
    bool ok = false;
    std::vector<size_t> limit; // limit[k - 1]: the largest shared-memory size with >= k CTAs
};

} // namespace

int occupancy(const void *fn, int nthreads, size_t smem)
{
    static std::mutex mu;
    static std::map<std::tuple<int, const void *, int>, OccTable> tables;
    if (smem > kSmemMax || nthreads <= 0) return 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_tuple(dev, fn, nthreads);
    auto it = tables.find(key);
    if (it == tables.end()) {
        OccTable t;
        auto query = [&](size_t s, int *occ) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, fn, nthreads, s) != cudaSuccess) {
                cudaGetLastError();
                return false;
            }
            return true;
        };
        int top = 0;
        t.ok = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSmemMax)) == cudaSuccess &&
               query(0, &top);
        if (!t.ok) cudaGetLastError();
        for (int k = 1; t.ok && k <= top; ++k) {
            // largest s in [0, kSmemMax] with occupancy(s) >= k (occupancy(0) >= k)
            size_t lo = 0, hi = kSmemMax;
            int o = 0;
            if (!query(hi, &o)) {
                t.ok = false;
                break;
            }
            if (o >= k) {
                lo = hi;
            } else {
                while (hi - lo > 1) {
                    const size_t mid = lo + (hi - lo) / 2;
                    if (!query(mid, &o)) {
                        t.ok = false;
                        break;
                    }
                    if (o >= k)
                        lo = mid;
                    else
                        hi = mid;
                }
            }
            t.limit.push_back(lo);
        }
        it = tables.emplace(key, t).first;
    }
    if (!it->second.ok) return 0;
    int n = 0;
    for (const size_t l : it->second.limit) n += smem <= l ? 1 : 0;
    return n;
}

} // namespace rs
