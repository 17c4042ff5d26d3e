// eap_dp_erp.cu -- instantiates the warp-per-pair DP and the diagonal upper
// bound for ERP (Eq. ERP, windowed).
#include "eap_internal.h"

namespace eaph {
using namespace eapd;

int launch_dp_erp(const LaunchCtx& c, bool ub_only) {
    return c.cost == 0 ? run_kind<FErp<0>, true>(c, ub_only) : run_kind<FErp<1>, true>(c, ub_only);
}

}  // namespace eaph
