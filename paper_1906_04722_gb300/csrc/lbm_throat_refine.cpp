// lbm_throat_refine.cpp -- entry pressures resolved below the ladder step
// (host code around two lbm_run_throat_batch calls).
//
// A throat's p_c^e is the largest bulk capillary pressure reached up to the
// increment at which it is invaded (Sec. 2.2.2), so a ladder resolves it only
// to one ladder step.  The refinement runs the ladder a second time on every
// throat invaded at increment k >= 1: the same levels up to k - 1 (the same
// steps, hence the same state: the run is deterministic), then n_fine equal
// sub-steps from level k - 1 to level k, each with the schedule's steps per
// increment, and reads p_c^e off that run.
#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "lbm_internal.h"

using namespace lbmk;

extern "C" {

int lbm_run_throat_batch_refined(const double* throats, int n, const lbm_params* params, const lbm_schedule* sched,
                                 int n_fine, lbm_throat_result* results, lbm_increment* rows, double* p_ce_fine,
                                 void* stream) {
    if (!throats || !params || !sched || !results || !rows || !p_ce_fine || n < 0 || n_fine < 1 || !sched->rho_in_nw ||
        sched->n_incr < 1) {
        set_error("lbm_run_throat_batch_refined: NULL argument, n < 0, n_fine < 1 or an empty ladder");
        return LBM_ERR_ARG;
    }
    int rc = lbm_run_throat_batch(throats, n, params, sched, results, rows, stream);
    if (rc) return rc;
    const int ni = sched->n_incr;
    auto level = [&](int t, int i) { return sched->rho_in_nw[(sched->per_throat ? (size_t)t * ni : 0) + i]; };
    try {
        std::vector<int> sel;
        int kmax = 0;
        for (int t = 0; t < n; ++t) {
            p_ce_fine[t] = results[t].p_ce;
            const int k = results[t].invaded_at;
            if (k >= 1) {
                sel.push_back(t);
                kmax = std::max(kmax, k);
            }
        }
        if (sel.empty() || n_fine == 1) return LBM_OK;
        const int m = (int)sel.size();
        const int K = kmax + n_fine;  // every fine ladder padded with its last level
        std::vector<double> sub((size_t)m * 12), lad((size_t)m * K);
        for (int q = 0; q < m; ++q) {
            const int t = sel[q], k = results[t].invaded_at;
            std::copy(throats + 12 * (size_t)t, throats + 12 * (size_t)t + 12, sub.begin() + 12 * (size_t)q);
            double* L = lad.data() + (size_t)q * K;
            for (int i = 0; i < k; ++i) L[i] = level(t, i);
            const double a = level(t, k - 1), b = level(t, k);
            for (int j = 1; j <= n_fine; ++j) L[k - 1 + j] = a + (b - a) * j / n_fine;
            for (int i = k + n_fine; i < K; ++i) L[i] = b;
        }
        lbm_schedule s2 = *sched;
        s2.n_incr = K;
        s2.rho_in_nw = lad.data();
        s2.per_throat = 1;
        std::vector<lbm_throat_result> res2(m);
        std::vector<lbm_increment> rows2((size_t)m * K);
        rc = lbm_run_throat_batch(sub.data(), m, params, &s2, res2.data(), rows2.data(), stream);
        if (rc) return rc;
        for (int q = 0; q < m; ++q)
            if (res2[q].invaded_at >= 0) p_ce_fine[sel[q]] = res2[q].p_ce;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return LBM_ERR_OOM;
    }
    return LBM_OK;
}

}  // extern "C"
