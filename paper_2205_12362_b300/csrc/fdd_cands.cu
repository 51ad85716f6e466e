// fdd_cands.cu -- helpers on candidate lists.
#include <algorithm>
#include <tuple>

#include "fdd_plan_impl.h"

using namespace fdd::host;

extern "C" {

int fdd_sort_candidates(fdd_candidate* cands, int64_t n) {
    if (n < 0 || (n > 0 && !cands)) return fail(FDD_ERR_INVALID_ARG, "bad argument");
    std::sort(cands, cands + n, [](const fdd_candidate& a, const fdd_candidate& b) {
        return std::tie(a.sb, a.dm_index, a.width_native, a.t_native) <
               std::tie(b.sb, b.dm_index, b.width_native, b.t_native);
    });
    return FDD_OK;
}

}  // extern "C"
