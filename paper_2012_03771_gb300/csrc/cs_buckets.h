// Layout of the hit buckets (host code): when the three-gap walk writes its
// stored hits as records per band of rows instead of clearing them directly,
// how many rows a band holds, how many records each (walk CTA, band) region
// holds, and after which large-prime chunks the records are cleared.
//
// A scattered atomic AND per stored hit costs a DRAM sector read and written
// back (about 100 bytes) once the bitset no longer fits in L2, while a record
// costs 4 bytes written and read and is cleared band after band with the band's
// words in L2.  So the automatic choice buckets bitsets of 256 MiB and more
// (twice L2) and keeps a band to at most a fifth of L2 (the apply kernel keeps
// about 1.3 bands in work beside its stream of records).
#pragma once
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

namespace cs {

// most bands of rows: 16 KB of per-band counters in a walking CTA
constexpr uint32_t BKT_MAX_BANDS = 4096;

struct BucketLayout {
    bool on = false;
    uint32_t band_log = 0;      // rows per band = 2^band_log
    uint64_t n_bands = 0;
    uint64_t n_regions = 0;     // regions per band: one per walk CTA
    uint64_t cap = 0;           // records per region, a multiple of 4
    bool bad_band_log = false;  // an explicit band_rows_log gives records above 32 bits or too many bands
};

// hit_buckets: 0 automatic, 1 off, 2 on; band_rows_log and bucket_records: 0
// automatic.  three_gap: the walk that can bucket; M_c rows of wpr 64-bit
// words; l2 bytes of L2; walk_ctas: CTAs of the walk's grid.
inline BucketLayout bucket_layout(uint32_t hit_buckets, uint32_t band_rows_log, uint64_t bucket_records,
                                  bool three_gap, bool have_chunks, uint64_t M_c, uint64_t wpr, uint64_t l2,
                                  uint64_t walk_ctas) {
    BucketLayout b;
    const uint64_t bitset_bytes = M_c * wpr * 8;
    bool on = hit_buckets == 2 || (hit_buckets == 0 && bitset_bytes >= (256ull << 20));
    on = on && three_gap && have_chunks && M_c > 0 && wpr > 0;
    uint32_t bl = band_rows_log;
    if (on && !bl) {
        const uint64_t band_max = l2 / 5;
        while ((2ull << bl) * wpr * 8 <= band_max && (2ull << bl) <= M_c) bl++;
        while (((M_c + (1ull << bl) - 1) >> bl) > BKT_MAX_BANDS) bl++;
    }
    // a record, (row in band) * 64 wpr + column, must fit 32 bits
    const bool fits = ((64ull * wpr) << bl) <= (1ull << 32);
    const uint64_t n_bands = (M_c + (1ull << bl) - 1) >> bl;
    b.bad_band_log = on && band_rows_log && (!fits || n_bands > BKT_MAX_BANDS);
    on = on && fits && n_bands <= BKT_MAX_BANDS;
    if (!on) return b;
    uint64_t cap = bucket_records;
    if (!cap) {
        // up to 8 GiB of records, at most twice the bitset (and at least 64 MiB)
        const uint64_t budget = std::min<uint64_t>(8ull << 30, std::max<uint64_t>(64ull << 20, 2 * bitset_bytes));
        cap = budget / 4 / (n_bands * walk_ctas);
    }
    // a multiple of 4, so that every region starts on a 16-byte boundary
    cap = std::min<uint64_t>(std::max<uint64_t>((cap + 3) / 4 * 4, 4), 1ull << 24);
    b.on = true;
    b.band_log = bl;
    b.n_bands = n_bands;
    b.n_regions = walk_ctas;
    b.cap = cap;
    return b;
}

// Expected stored hits of primes in (lo, hi] over M_c rows of W stored
// columns: M_c W sum 1/p, by Mertens' second theorem log log hi - log log lo.
inline double expected_stored_hits(uint64_t lo, uint64_t hi, uint64_t M_c, uint64_t W) {
    const double l = std::max<double>((double)lo, 3.0);
    const double h = std::max<double>((double)hi, l);
    return (double)M_c * (double)W * std::log(std::log(h) / std::log(l));
}

// apply_after[c] = 1 when the records are cleared after chunk c's walk: chunks
// are grouped in order so that a group's expected stored hits fill at most
// 60% of all regions (a chunk that alone expects more forms its own group, and
// its overflow clears directly); the last chunk always ends a group.
inline std::vector<uint8_t> apply_groups(const std::vector<std::pair<uint64_t, uint64_t>> &chunks, uint64_t M_c,
                                         uint64_t W, const BucketLayout &b) {
    std::vector<uint8_t> after(chunks.size(), 0);
    if (chunks.empty()) return after;
    const double room = 0.6 * (double)b.cap * (double)b.n_regions * (double)b.n_bands;
    double acc = 0;
    for (size_t c = 0; c < chunks.size(); c++) {
        const double e = expected_stored_hits(chunks[c].first, chunks[c].second, M_c, W);
        if (c > 0 && acc > 0 && acc + e > room) {
            after[c - 1] = 1;
            acc = 0;
        }
        acc += e;
    }
    after[chunks.size() - 1] = 1;
    return after;
}

}  // namespace cs
