// Host build of the hit-bucket layout (csrc/cs_buckets.h) for CPU tests: reads
// lines "hit_buckets band_rows_log bucket_records three_gap M_c wpr W l2
// walk_ctas n lo_1 hi_1 ... lo_n hi_n" and prints "on band_log n_bands n_regions
// cap bad_band_log a_1 ... a_n" (a_c = 1 when the records are cleared after
// chunk c).
#include <cstdio>
#include <cstdint>
#include <utility>
#include <vector>

#include "../../paper_2012_03771_gb300/csrc/cs_buckets.h"

int main() {
    unsigned hb, bl, three_gap;
    unsigned long long recs, M_c, wpr, W, l2, ctas, n;
    while (scanf("%u %u %llu %u %llu %llu %llu %llu %llu %llu", &hb, &bl, &recs, &three_gap, &M_c, &wpr, &W, &l2,
                 &ctas, &n) == 10) {
        std::vector<std::pair<uint64_t, uint64_t>> chunks(n);
        for (auto &c : chunks) {
            unsigned long long lo, hi;
            if (scanf("%llu %llu", &lo, &hi) != 2) return 1;
            c = {lo, hi};
        }
        const cs::BucketLayout b = cs::bucket_layout(hb, bl, recs, three_gap != 0, !chunks.empty(), M_c, wpr, l2, ctas);
        printf("%d %u %llu %llu %llu %d", b.on ? 1 : 0, b.band_log, (unsigned long long)b.n_bands,
               (unsigned long long)b.n_regions, (unsigned long long)b.cap, b.bad_band_log ? 1 : 0);
        if (b.on)
            for (uint8_t a : cs::apply_groups(chunks, M_c, W, b)) printf(" %u", (unsigned)a);
        printf("\n");
    }
    return 0;
}
