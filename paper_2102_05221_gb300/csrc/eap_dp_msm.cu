// eap_dp_msm.cu -- instantiates the warp-per-pair DP and the diagonal upper
// bound for MSM (Eq. MSM with Eq. MSMCost).
#include "eap_internal.h"

namespace eaph {
using namespace eapd;

int launch_dp_msm(const LaunchCtx& c, bool ub_only) {
    return run_kind<FMsm, false>(c, ub_only);
}

}  // namespace eaph
