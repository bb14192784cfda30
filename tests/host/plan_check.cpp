// Host build of the plan's m-class tiers (csrc/cs_classes.h) for CPU tests:
// reads "three_gap d M_start M_inc S m_classes class_min_hits class_item_hits lo"
// lines and prints, for a large-prime chunk whose primes start above lo, the
// classes its walk takes: "Q n items r_1 ... r_n" (the residues of m - M_start
// mod Q that are walked).
#include <cstdio>
#include <cstdint>

#include "../../paper_2012_03771_gb300/csrc/cs_classes.h"

int main() {
    unsigned three_gap, m_classes, min_hits, item_hits;
    unsigned long long d, M_start, M_inc, S, lo;
    while (scanf("%u %llu %llu %llu %llu %u %u %u %llu", &three_gap, &d, &M_start, &M_inc, &S, &m_classes,
                 &min_hits, &item_hits, &lo) == 9) {
        cs_tuning t{};
        t.m_classes = m_classes;
        t.class_min_hits = min_hits;
        t.class_item_hits = item_hits;
        const cs::ClassTiers tiers = cs::class_tiers(three_gap != 0, d, M_start, M_inc, S, t);
        const cs::MClasses mc = tiers.for_chunk(lo);
        printf("%u %u %u", mc.Q, mc.n, mc.items);
        for (uint32_t k = 0; k < mc.n; k++) printf(" %u", mc.items ? (unsigned)mc.item_off[k] : mc.off[k]);
        printf("\n");
    }
    return 0;
}
