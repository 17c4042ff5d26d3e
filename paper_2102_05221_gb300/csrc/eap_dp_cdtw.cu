// eap_dp_cdtw.cu -- instantiates the warp-per-pair DP and the diagonal upper
// bound for CDTW (Eq. DTW inside the Sakoe-Chiba window, Section 2.3.2).
#include "eap_internal.h"

namespace eaph {
using namespace eapd;

int launch_dp_cdtw(const LaunchCtx& c, bool ub_only) {
    return c.cost == 0 ? run_kind<FDtw<0>, true>(c, ub_only) : run_kind<FDtw<1>, true>(c, ub_only);
}

}  // namespace eaph
