// eap_dp_twe.cu -- instantiates the warp-per-pair DP and the diagonal upper
// bound for TWE (Eq. TWE with Eq. TWECost).
#include "eap_internal.h"

namespace eaph {
using namespace eapd;

int launch_dp_twe(const LaunchCtx& c, bool ub_only) {
    return c.cost == 0 ? run_kind<FTwe<0>, false>(c, ub_only) : run_kind<FTwe<1>, false>(c, ub_only);
}

}  // namespace eaph
