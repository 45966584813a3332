// lbm_throat_surrogate.cpp -- the throat surrogate behind the C ABI (host code
// around the tensor-core network of lbm_mlp.cu and the batched LBM of
// lbm_batch.cu).
//
// The hybrid method reads, for every pore throat, the entry capillary pressure
// p_c^e and the throat's drainage curve off one LBM run (Sec. 2.2.2).  The
// surrogate learns that map on throats the batched LBM has run and answers new
// throats with an ensemble; throats on which the members disagree by more than
// a relative spread go back to the batched LBM.
//
// Inputs per throat (LBM_SURROGATE_INPUTS = 24): the three radii and the three
// centre distances over the mean radius R (spheres ordered by decreasing
// radius, ties in input order), the contact angle (7); the lattice description
// of the throat box (lbm_throat_lattice_features, 14); its narrowest section's
// equivalent radius and lattice incircles over R (3).  Outputs (1 + n_incr):
// p_c^e R and the throat's S_w after each increment.  Inputs and targets are
// standardised by their training means and standard deviations.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "lbm_internal.h"

struct lbm_throat_surrogate {
    lbm_throat_surrogate_config cfg;
    lbm_surrogate* net;
    void* stream;
    int n_out;
    bool fitted;
    std::vector<double> x_mu, x_sd, y_mu, y_sd;
};

namespace lbmk {
namespace {

constexpr int NIN = LBM_SURROGATE_INPUTS;

// The 7 geometric inputs and the mean radius of one throat.
void geometric_inputs(const double* t, double theta, double* x, double* R_out) {
    int order[3] = {0, 1, 2};
    std::stable_sort(order, order + 3, [&](int a, int b) { return t[4 * a + 3] > t[4 * b + 3]; });
    double c[3][3], r[3];
    for (int i = 0; i < 3; ++i) {
        for (int d = 0; d < 3; ++d) c[i][d] = t[4 * order[i] + d];
        r[i] = t[4 * order[i] + 3];
    }
    const double R = (r[0] + r[1] + r[2]) / 3.0;
    auto dist = [&](int a, int b) {
        const double dx = c[a][0] - c[b][0], dy = c[a][1] - c[b][1], dz = c[a][2] - c[b][2];
        return std::sqrt(dx * dx + dy * dy + dz * dz);
    };
    x[0] = r[0] / R;
    x[1] = r[1] / R;
    x[2] = r[2] / R;
    x[3] = dist(0, 1) / R;
    x[4] = dist(1, 2) / R;
    x[5] = dist(0, 2) / R;
    x[6] = theta;
    *R_out = R;
}

int inputs(const double* throats, int n, double theta, std::vector<double>& X, std::vector<double>& R) {
    X.assign((size_t)n * NIN, 0.0);
    R.assign((size_t)n, 0.0);
    std::vector<double> L((size_t)n * LBM_THROAT_LATTICE_FEATURES);
    int rc = lbm_throat_lattice_features(throats, n, L.data());
    if (rc) return rc;
    for (int i = 0; i < n; ++i) {
        double* x = X.data() + (size_t)i * NIN;
        double Ri;
        geometric_inputs(throats + 12 * (size_t)i, theta, x, &Ri);
        R[(size_t)i] = Ri;
        const double* l = L.data() + (size_t)i * LBM_THROAT_LATTICE_FEATURES;
        for (int k = 0; k < LBM_THROAT_LATTICE_FEATURES; ++k) x[7 + k] = l[k];
        x[21] = l[5] / Ri;
        x[22] = l[8] / Ri;
        x[23] = l[9] / Ri;
    }
    return LBM_OK;
}

void moments(const std::vector<double>& A, int n, int w, std::vector<double>& mu, std::vector<double>& sd) {
    mu.assign((size_t)w, 0.0);
    sd.assign((size_t)w, 0.0);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < w; ++k) mu[(size_t)k] += A[(size_t)i * w + k];
    for (int k = 0; k < w; ++k) mu[(size_t)k] /= n;
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < w; ++k) {
            const double d = A[(size_t)i * w + k] - mu[(size_t)k];
            sd[(size_t)k] += d * d;
        }
    for (int k = 0; k < w; ++k) sd[(size_t)k] = std::sqrt(sd[(size_t)k] / n) + 1e-6;
}

bool valid_throats(const double* t, int n) {
    for (long long i = 0; i < 12LL * n; ++i)
        if (!std::isfinite(t[i]) || (i % 4 == 3 && !(t[i] > 0))) return false;
    return true;
}

// p_c^e, its relative ensemble spread and (optionally) the curves of n throats.
int predict(lbm_throat_surrogate* ts, const double* throats, int n, double* pce, double* rel, float* curves) {
    std::vector<double> X, R;
    int rc = inputs(throats, n, ts->cfg.theta, X, R);
    if (rc) return rc;
    std::vector<float> Xn((size_t)n * NIN);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < NIN; ++k)
            Xn[(size_t)i * NIN + k] = (float)((X[(size_t)i * NIN + k] - ts->x_mu[(size_t)k]) / ts->x_sd[(size_t)k]);
    const int no = ts->n_out;
    std::vector<float> mean((size_t)n * no), spread((size_t)n * no);
    rc = lbm_surrogate_predict(ts->net, Xn.data(), n, mean.data(), spread.data());
    if (rc) return rc;
    for (int i = 0; i < n; ++i) {
        const double m0 = mean[(size_t)i * no] * ts->y_sd[0] + ts->y_mu[0];
        const double s0 = spread[(size_t)i * no] * ts->y_sd[0];
        pce[i] = m0 / R[(size_t)i];
        if (rel) rel[i] = std::fabs(s0) / std::max(std::fabs(m0), 1e-12);
        if (curves)
            for (int k = 1; k < no; ++k)
                curves[(size_t)i * (no - 1) + (k - 1)] =
                    (float)(mean[(size_t)i * no + k] * ts->y_sd[(size_t)k] + ts->y_mu[(size_t)k]);
    }
    return LBM_OK;
}

}  // namespace
}  // namespace lbmk

using namespace lbmk;

extern "C" {

int lbm_contact_angle_estimate(double G_ads_w, double G_ads_nw, double G, double rho_major, double rho_minor,
                               double* theta_out) {
    if (!theta_out || !(G > 0) || !(rho_major > rho_minor)) {
        set_error("lbm_contact_angle_estimate: needs G > 0, rho_major > rho_minor and an output");
        return LBM_ERR_ARG;
    }
    const double c = (G_ads_nw - G_ads_w) / (G * (rho_major - rho_minor) / 2.0);
    *theta_out = std::acos(std::max(-1.0, std::min(1.0, c)));
    return LBM_OK;
}

int lbm_pressure_ladder(const double* r_in, int n, int n_incr, double lo, double hi, double rho_major,
                        double rho_minor, double G, double* out) {
    if (!r_in || !out || n < 0 || n_incr < 1 || !std::isfinite(lo) || !std::isfinite(hi)) {
        set_error("lbm_pressure_ladder: NULL argument, n < 0 or n_incr < 1");
        return LBM_ERR_ARG;
    }
    // p_c,res = (rho_in - rho_major)(1 + G rho_minor)/3 at rest (Eq. 5 on the
    // inlet and outlet layers), so rho_in = rho_major + 3 p_c / (1 + G rho_minor)
    for (int i = 0; i < n; ++i) {
        const double r = std::max(r_in[i], 0.5);
        for (int k = 0; k < n_incr; ++k) {
            const double pc = (n_incr == 1 ? lo : lo + (hi - lo) * k / (double)(n_incr - 1)) / r;
            out[(size_t)i * n_incr + k] = rho_major + 3.0 * pc / (1.0 + G * rho_minor);
        }
    }
    return LBM_OK;
}

int lbm_throat_surrogate_inputs(const double* throats, int n, double theta, float* X_out, double* R_out) {
    if (!throats || !X_out || n < 1 || !std::isfinite(theta) || !valid_throats(throats, n)) {
        set_error("lbm_throat_surrogate_inputs: bad throats, n < 1 or non-finite theta");
        return LBM_ERR_ARG;
    }
    try {
        std::vector<double> X, R;
        int rc = inputs(throats, n, theta, X, R);
        if (rc) return rc;
        for (size_t i = 0; i < X.size(); ++i) X_out[i] = (float)X[i];
        if (R_out)
            for (int i = 0; i < n; ++i) R_out[i] = R[(size_t)i];
        return LBM_OK;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return LBM_ERR_OOM;
    }
}

int lbm_throat_surrogate_create(const lbm_throat_surrogate_config* cfg, void* stream, lbm_throat_surrogate** out) {
    if (!cfg || !out || cfg->n_incr < 1 || !std::isfinite(cfg->theta)) {
        set_error("lbm_throat_surrogate_create: NULL argument, n_incr < 1 or non-finite theta");
        return LBM_ERR_ARG;
    }
    lbm_throat_surrogate* ts = new (std::nothrow) lbm_throat_surrogate();
    if (!ts) { set_error("host allocation failed"); return LBM_ERR_OOM; }
    ts->cfg = *cfg;
    ts->stream = stream;
    ts->n_out = 1 + cfg->n_incr;
    ts->fitted = false;
    ts->net = nullptr;
    lbm_surrogate_config sc;
    sc.n_in = NIN;
    sc.n_hidden = cfg->n_hidden;
    sc.n_layers = cfg->n_layers;
    sc.n_out = ts->n_out;
    sc.n_members = cfg->n_members;
    sc.half = cfg->half;
    sc.seed = cfg->seed;
    int rc = lbm_surrogate_create(&sc, stream, &ts->net);
    if (rc) {
        delete ts;
        return rc;
    }
    *out = ts;
    return LBM_OK;
}

int lbm_throat_surrogate_fit(lbm_throat_surrogate* ts, const double* throats, int n, const lbm_throat_result* results,
                             const lbm_increment* rows, int epochs, int batch, float lr, unsigned long long shuffle_seed,
                             double* epoch_loss, int* n_used) {
    if (!ts || !throats || !results || !rows || n < 1 || !valid_throats(throats, n)) {
        set_error("lbm_throat_surrogate_fit: NULL argument, n < 1 or bad throats");
        return LBM_ERR_ARG;
    }
    try {
        std::vector<double> X, R;
        int rc = inputs(throats, n, ts->cfg.theta, X, R);
        if (rc) return rc;
        // throats invaded within the ladder carry a target
        const int ni = ts->cfg.n_incr, no = ts->n_out;
        std::vector<double> Xu, Yu;
        for (int i = 0; i < n; ++i) {
            if (!std::isfinite(results[i].p_ce)) continue;
            Xu.insert(Xu.end(), X.begin() + (size_t)i * NIN, X.begin() + (size_t)(i + 1) * NIN);
            Yu.push_back(results[i].p_ce * R[(size_t)i]);
            for (int k = 0; k < ni; ++k) Yu.push_back(rows[(size_t)i * ni + k].S_w);
        }
        const int m = (int)(Xu.size() / NIN);
        if (n_used) *n_used = m;
        if (m < 2) { set_error("lbm_throat_surrogate_fit: fewer than two invaded throats"); return LBM_ERR_ARG; }
        moments(Xu, m, NIN, ts->x_mu, ts->x_sd);
        moments(Yu, m, no, ts->y_mu, ts->y_sd);
        std::vector<float> Xn(Xu.size()), Yn(Yu.size());
        for (int i = 0; i < m; ++i) {
            for (int k = 0; k < NIN; ++k)
                Xn[(size_t)i * NIN + k] = (float)((Xu[(size_t)i * NIN + k] - ts->x_mu[(size_t)k]) / ts->x_sd[(size_t)k]);
            for (int k = 0; k < no; ++k)
                Yn[(size_t)i * no + k] = (float)((Yu[(size_t)i * no + k] - ts->y_mu[(size_t)k]) / ts->y_sd[(size_t)k]);
        }
        rc = lbm_surrogate_train(ts->net, Xn.data(), Yn.data(), m, epochs, batch, lr, shuffle_seed, epoch_loss);
        if (rc) return rc;
        ts->fitted = true;
        return LBM_OK;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return LBM_ERR_OOM;
    }
}

int lbm_throat_surrogate_predict(lbm_throat_surrogate* ts, const double* throats, int n, double* p_ce,
                                 double* rel_spread, float* curves) {
    if (!ts || !throats || !p_ce || n < 1 || !valid_throats(throats, n)) {
        set_error("lbm_throat_surrogate_predict: NULL argument, n < 1 or bad throats");
        return LBM_ERR_ARG;
    }
    if (!ts->fitted) { set_error("lbm_throat_surrogate_predict: not fitted"); return LBM_ERR_STATE; }
    try {
        return predict(ts, throats, n, p_ce, rel_spread, curves);
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return LBM_ERR_OOM;
    }
}

int lbm_throat_surrogate_predict_with_fallback(lbm_throat_surrogate* ts, const double* throats, int n,
                                               double spread_tol, const lbm_params* params,
                                               const lbm_schedule* sched, double* p_ce, int* used_lbm,
                                               double* seconds) {
    if (!ts || !throats || !p_ce || !used_lbm || !params || !sched || n < 1 || !(spread_tol >= 0) ||
        !valid_throats(throats, n) || !sched->rho_in_nw || sched->n_incr < 1) {
        set_error("lbm_throat_surrogate_predict_with_fallback: bad argument");
        return LBM_ERR_ARG;
    }
    if (!ts->fitted) { set_error("lbm_throat_surrogate_predict_with_fallback: not fitted"); return LBM_ERR_STATE; }
    try {
        using clk = std::chrono::steady_clock;
        const auto t0 = clk::now();
        std::vector<double> rel((size_t)n);
        int rc = predict(ts, throats, n, p_ce, rel.data(), nullptr);
        if (rc) return rc;
        const auto t1 = clk::now();
        // the spread rule: throats whose members disagree go to the batched LBM
        std::vector<int> fall;
        for (int i = 0; i < n; ++i) {
            used_lbm[i] = rel[(size_t)i] > spread_tol ? 1 : 0;
            if (used_lbm[i]) fall.push_back(i);
        }
        if (!fall.empty()) {
            const int nf = (int)fall.size(), ni = sched->n_incr;
            std::vector<double> sub((size_t)nf * 12);
            std::vector<double> lad;
            for (int j = 0; j < nf; ++j)
                std::copy(throats + 12 * (size_t)fall[(size_t)j], throats + 12 * (size_t)(fall[(size_t)j] + 1),
                          sub.begin() + 12 * (size_t)j);
            lbm_schedule s2 = *sched;
            if (sched->per_throat) {
                lad.resize((size_t)nf * ni);
                for (int j = 0; j < nf; ++j)
                    std::copy(sched->rho_in_nw + (size_t)fall[(size_t)j] * ni,
                              sched->rho_in_nw + (size_t)(fall[(size_t)j] + 1) * ni, lad.begin() + (size_t)j * ni);
                s2.rho_in_nw = lad.data();
            }
            std::vector<lbm_throat_result> res((size_t)nf);
            std::vector<lbm_increment> rows((size_t)nf * ni);
            rc = lbm_run_throat_batch(sub.data(), nf, params, &s2, res.data(), rows.data(), ts->stream);
            if (rc) return rc;
            for (int j = 0; j < nf; ++j) p_ce[fall[(size_t)j]] = res[(size_t)j].p_ce;
        }
        const auto t2 = clk::now();
        if (seconds) {
            seconds[0] = std::chrono::duration<double>(t1 - t0).count();
            seconds[1] = std::chrono::duration<double>(t2 - t1).count();
        }
        return LBM_OK;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return LBM_ERR_OOM;
    }
}

int lbm_throat_surrogate_scaling(const lbm_throat_surrogate* ts, double* x_mu, double* x_sd, double* y_mu,
                                 double* y_sd) {
    if (!ts || !x_mu || !x_sd || !y_mu || !y_sd) { set_error("NULL argument"); return LBM_ERR_ARG; }
    if (!ts->fitted) { set_error("lbm_throat_surrogate_scaling: not fitted"); return LBM_ERR_STATE; }
    std::copy(ts->x_mu.begin(), ts->x_mu.end(), x_mu);
    std::copy(ts->x_sd.begin(), ts->x_sd.end(), x_sd);
    std::copy(ts->y_mu.begin(), ts->y_mu.end(), y_mu);
    std::copy(ts->y_sd.begin(), ts->y_sd.end(), y_sd);
    return LBM_OK;
}

lbm_surrogate* lbm_throat_surrogate_network(lbm_throat_surrogate* ts) { return ts ? ts->net : nullptr; }

void lbm_throat_surrogate_destroy(lbm_throat_surrogate* ts) {
    if (!ts) return;
    lbm_surrogate_destroy(ts->net);
    delete ts;
}

}  // extern "C"
