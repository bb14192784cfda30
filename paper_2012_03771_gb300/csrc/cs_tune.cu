// Autotuner for the small/large prime threshold T, the tile height and the
// size of the large-prime walk's work items (expected walked hits per item,
// i.e. how many primes and m-segments a CTA's warps take at a time).
//
// Section 3.2 leaves the threshold open ("naively p > 10 S"; the runtime
// model's C_mult is about 50).  Here it trades two kernels: the tile sieve costs
// about M_c per small prime, the walk about M_inc S / p hits plus a few solves
// per large prime.  Both grow with M_inc at the same rate, so the best T hardly
// depends on M_inc; it depends on S, on the primes near T and on the GPU.  The
// tuner therefore times candidate settings on a proxy with the same P, d and SL,
// M_inc clipped to 1e5 and L to 1e9 (a few tens of milliseconds per run): first
// T and the tile height together, then the item size for the winner.  The
// choice is kept per (P, d, SL, ceil(log2 L)) in memory and, if a path is
// given, in a text file that later processes read back (lines of six fields,
// without an item size, mean the automatic one).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/combsieve.h"
#include "cs_internal.h"

using namespace cs;

namespace {

using Key = std::tuple<uint32_t, uint64_t, uint32_t, uint32_t>;   // P, d, SL, ceil(log2 L)
struct Choice {
    uint64_t T_over_S_x100;   // threshold as a multiple of S, times 100
    uint32_t tile_rows;
    uint32_t item_hits;       // walked hits per work item (0: the automatic 128)
};

std::mutex g_mu;
std::map<Key, Choice> g_mem;

uint32_t log2_ceil(uint64_t x) {
    uint32_t k = 0;
    while (k < 63 && (1ull << k) < x) k++;
    return k;
}

void load_file(const char *path) {
    FILE *f = fopen(path, "r");
    if (!f) return;
    char line[256];
    while (fgets(line, sizeof(line), f)) {
        unsigned P, SL, lg, rows, items = 0;
        unsigned long long d, tx;
        const int n = sscanf(line, "%u %llu %u %u %llu %u %u", &P, &d, &SL, &lg, &tx, &rows, &items);
        if (n == 6 || n == 7) g_mem[Key{P, d, SL, lg}] = Choice{tx, rows, n == 7 ? items : 0u};
    }
    fclose(f);
}

void append_file(const char *path, const Key &k, const Choice &c) {
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%u %llu %u %u %llu %u %u\n", std::get<0>(k), (unsigned long long)std::get<1>(k), std::get<2>(k),
            std::get<3>(k), (unsigned long long)c.T_over_S_x100, c.tile_rows, c.item_hits);
    fclose(f);
}

// device time of one sieve of the proxy (median of five after one warm-up run),
// or a negative value
double time_once(uint32_t P, uint64_t d, uint64_t M_start, uint64_t M_inc, uint32_t SL, uint64_t L,
                 const cs_tuning &t, cudaStream_t st) {
    cs_plan_t plan = nullptr;
    if (cs_plan(P, d, M_start, M_inc, SL, L, &t, &plan)) return -1;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    std::vector<float> ts;
    for (int rep = 0; rep < 6; rep++) {
        cudaEventRecord(a, st);
        if (cs_sieve(plan, st)) break;
        cudaEventRecord(b, st);
        if (cudaEventSynchronize(b) != cudaSuccess) break;
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0) ts.push_back(ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cs_destroy(plan);
    if (ts.size() < 5) return -1;
    std::sort(ts.begin(), ts.end());
    return ts[ts.size() / 2];
}

}  // namespace

extern "C" cs_status cs_autotune(uint32_t P, uint64_t d, uint64_t M_start, uint64_t M_inc, uint32_t SL,
                                 uint64_t L, const char *cache_path, cs_tuning *out) {
    if (!out) return set_error(CS_EINVAL, "out is NULL");
    cs_status s = validate_params(P, d, M_start, M_inc, SL, L);
    if (s) return s;
    memset(out, 0, sizeof(*out));
    out->large_mode = 2;
    const uint64_t S = 2ull * SL + 1;
    const Key key{P, d, SL, log2_ceil(std::max<uint64_t>(L, 2))};
    std::lock_guard<std::mutex> lk(g_mu);
    if (cache_path) load_file(cache_path);
    auto it = g_mem.find(key);
    if (it == g_mem.end()) {
        // proxy: same K and interval, fewer m, lower limit
        const uint64_t pM = std::min<uint64_t>(M_inc, 100000), pL = std::min<uint64_t>(L, 1000000000ull);
        const uint64_t mults_x100[] = {200, 250, 300, 400, 500, 600, 800, 1000, 1200, 1600};
        const uint32_t rows[] = {8, 16, 32};
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
            return set_error(CS_EDEVICE, "cudaStreamCreate");
        double best = -1;
        Choice pick{800, 0, 0};
        for (uint64_t mx : mults_x100)
            for (uint32_t tr : rows) {
                cs_tuning t{};
                t.large_mode = 2;
                t.tile_rows = tr;
                t.threshold = std::max<uint64_t>(S * mx / 100, 2ull * SL);
                if (t.threshold > (1ull << 30)) continue;
                double ms = time_once(P, d, M_start, pM, SL, pL, t, st);
                if (ms >= 0 && (best < 0 || ms < best)) {
                    best = ms;
                    pick = Choice{mx, tr, 0};
                }
            }
        if (best >= 0) {
            // work-item size for the chosen threshold and tile height (the
            // automatic 128 is the timing above)
            for (uint32_t ih : {32u, 64u, 256u, 512u}) {
                cs_tuning t{};
                t.large_mode = 2;
                t.tile_rows = pick.tile_rows;
                t.threshold = std::max<uint64_t>(S * pick.T_over_S_x100 / 100, 2ull * SL);
                t.item_hits = ih;
                double ms = time_once(P, d, M_start, pM, SL, pL, t, st);
                if (ms >= 0 && ms < best) {
                    best = ms;
                    pick.item_hits = ih;
                }
            }
        }
        cudaStreamDestroy(st);
        if (best < 0) return set_error(CS_EDEVICE, "autotune: no candidate ran");
        g_mem[key] = pick;
        if (cache_path) append_file(cache_path, key, pick);
        it = g_mem.find(key);
    }
    out->threshold = std::min<uint64_t>(std::max<uint64_t>(S * it->second.T_over_S_x100 / 100, 2ull * SL), 1ull << 30);
    out->tile_rows = it->second.tile_rows;
    out->item_hits = it->second.item_hits;
    return CS_OK;
}
