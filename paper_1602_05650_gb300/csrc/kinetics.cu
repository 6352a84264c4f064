// Two-state dynamic instability of the fibers' plus ends (Sec. 2.4 growth,
// Sec. 5 catastrophe and rescue; host code): the growth rates fs_set_growth
// takes, drawn from the per-fiber state with the caller's uniform random
// numbers.
#include <cmath>

#include "internal.h"

using namespace fs;

extern "C" {

fs_status fs_dynamic_instability(int32_t n, const fs_kinetics *k, double dt, const double *L, const double *u,
                                 int32_t *state, double *Ldot)
{
    if (n < 0 || !k || (n > 0 && (!L || !u || !state || !Ldot)) || !(dt > 0.0) || !std::isfinite(dt)) {
        set_error("fs_dynamic_instability: bad sizes, NULL arrays or dt not in (0, inf)");
        return FS_EINVAL;
    }
    // written so that NaN fails: speeds and rates finite and >= 0, lengths finite
    const double rates[4] = {k->v_grow, k->v_shrink, k->f_cat, k->f_res};
    for (double r : rates)
        if (!(r >= 0.0) || !std::isfinite(r)) {
            set_error("fs_dynamic_instability: speeds and rates must be finite and >= 0");
            return FS_EINVAL;
        }
    if (!std::isfinite(k->L_min) || !std::isfinite(k->L_max)) {
        set_error("fs_dynamic_instability: L_min and L_max must be finite");
        return FS_EINVAL;
    }
    const double p_cat = -std::expm1(-k->f_cat * dt);
    const double p_res = -std::expm1(-k->f_res * dt);
    for (int32_t i = 0; i < n; ++i) {
        int32_t s = state[i] ? 1 : 0;
        if (u[i] < (s ? p_cat : p_res)) s = 1 - s;           // catastrophe or rescue
        if (s == 0 && L[i] - k->v_shrink * dt < k->L_min) {
            s = 1;                                              // rescued at the minimum length
        } else if (s == 1 && k->L_max > 0.0 && L[i] + k->v_grow * dt > k->L_max) {
            s = 0;                                              // capped at the maximum length
        }
        state[i] = s;
        Ldot[i] = s ? k->v_grow : -k->v_shrink;
    }
    return FS_OK;
}

}  // extern "C"
