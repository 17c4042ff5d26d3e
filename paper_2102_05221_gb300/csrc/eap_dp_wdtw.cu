// eap_dp_wdtw.cu -- instantiates the warp-per-pair DP and the diagonal upper
// bound for WDTW (Eq. WDTW).
#include "eap_internal.h"

namespace eaph {
using namespace eapd;

int launch_dp_wdtw(const LaunchCtx& c, bool ub_only) {
    return c.cost == 0 ? run_kind<FWdtw<0>, false>(c, ub_only) : run_kind<FWdtw<1>, false>(c, ub_only);
}

}  // namespace eaph
