// Line-protocol driver of the serving engine's admission bookkeeping
// (paper_cs_0611109_gb300/csrc/rcg_admission.h) for the CPU tests.
//   I budget max_inflight              -> "ok"
//   R arrival footprint n lo hi [lo hi] -> "ok <id>"
//   A now                               -> "ok <admitted ids...>"
//   X id                                -> "ok"        (retire)
//   S                                   -> "ok <inflight> <budget used> <conflict waits>"
//   Q                                   -> quit
#include <stdint.h>
#include <stdio.h>

#include <memory>
#include <string>
#include <vector>

#include "rcg_admission.h"

int main() {
    std::unique_ptr<rcg::Admission> adm;
    char op[8];
    while (scanf("%7s", op) == 1) {
        const std::string o(op);
        if (o == "I") {
            unsigned long long budget, max_inflight;
            if (scanf("%llu %llu", &budget, &max_inflight) != 2) return 2;
            adm.reset(new rcg::Admission(budget, static_cast<uint32_t>(max_inflight)));
            printf("ok\n");
        } else if (o == "R") {
            unsigned long long arrival, footprint, n;
            if (scanf("%llu %llu %llu", &arrival, &footprint, &n) != 3 || n < 1 || n > 2) return 2;
            rcg::Admission::Item it;
            it.arrival_ns = arrival;
            it.footprint = footprint;
            it.n_ext = static_cast<uint32_t>(n);
            for (unsigned k = 0; k < n; ++k) {
                unsigned long long lo, hi;
                if (scanf("%llu %llu", &lo, &hi) != 2) return 2;
                it.ext[k].lo = static_cast<uintptr_t>(lo);
                it.ext[k].hi = static_cast<uintptr_t>(hi);
            }
            printf("ok %llu\n", static_cast<unsigned long long>(adm->add(it)));
        } else if (o == "A") {
            unsigned long long now;
            if (scanf("%llu", &now) != 1) return 2;
            std::vector<uint64_t> ids;
            adm->admit(now, [&](uint64_t id) { ids.push_back(id); });
            printf("ok");
            for (uint64_t id : ids) printf(" %llu", static_cast<unsigned long long>(id));
            printf("\n");
        } else if (o == "X") {
            unsigned long long id;
            if (scanf("%llu", &id) != 1) return 2;
            adm->retire(id);
            printf("ok\n");
        } else if (o == "S") {
            printf("ok %u %llu %llu\n", adm->inflight(), static_cast<unsigned long long>(adm->budget_used()),
                   static_cast<unsigned long long>(adm->conflict_waits()));
        } else if (o == "Q") {
            return 0;
        } else {
            return 2;
        }
        fflush(stdout);
    }
    return 0;
}
