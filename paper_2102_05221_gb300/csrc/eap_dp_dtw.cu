// eap_dp_dtw.cu -- instantiates the warp-per-pair DP and the diagonal upper
// bound for DTW (Eq. DTW, no window).
#include "eap_internal.h"

namespace eaph {
using namespace eapd;

int launch_dp_dtw(const LaunchCtx& c, bool ub_only) {
    return c.cost == 0 ? run_kind<FDtw<0>, false>(c, ub_only) : run_kind<FDtw<1>, false>(c, ub_only);
}

}  // namespace eaph
