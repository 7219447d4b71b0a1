// Sampling and resolution design figures of Sec. II-C/D for a polyline array
// (host code; no device work).
//
//   receive spacing   dd <= lambda_min sqrt((L_R + D)^2 / 4 + R_0^2) / (L_R + D)
//                     (multistatic receive subarray; half of it monostatic,
//                     two-way propagation; the transmit array is free)
//   scan step         dz' <= lambda_min / (4 sin(theta_z / 2))
//   resolutions       dx ~ lambda_c / (4 sin(theta_h / 2)),  dy = c / (2 B),
//                     dz = lambda_c / (4 sin(theta_z / 2))
//
// theta_h: angle of the circumscribed arc (all chords); theta_z: the smaller of
// the angle the scan length subtends from the scene centre at the array
// radius and the antenna beamwidth along the scan; L_R: chord length; R_0:
// distance from a chord to the scene centre; D: the largest target dimension.
#include <algorithm>
#include <cmath>

#include "../../include/polyline.h"
#include "common.cuh"
#include "kernels.h"

extern "C" pl_status pl_design(const pl_geometry *g, const pl_scan *s, const pl_freqs *f,
                               double target_dim, double beamwidth_z_deg, pl_design_info *out) {
    if (!g || !s || !f || !out) return pl_internal_fail(PL_ERR_ARG, "NULL argument");
    if (f->n < 1 || !f->f_hz) return pl_internal_fail(PL_ERR_FREQ, "no frequencies");
    if (!(g->radius > 0) || g->n_sections < 1 || !(g->chord_len > 0) ||
        g->chord_len > 2.0 * g->radius)
        return pl_internal_fail(PL_ERR_GEOMETRY, "radius, sections and chord length must describe a polyline on the circle");
    if (!(target_dim >= 0) || !(beamwidth_z_deg >= 0) || s->n < 1)
        return pl_internal_fail(PL_ERR_ARG, "target size, beamwidth and scan must be non-negative");
    double fmin = f->f_hz[0], fmax = f->f_hz[0];
    for (int m = 0; m < f->n; ++m) {
        if (!(f->f_hz[m] > 0)) return pl_internal_fail(PL_ERR_FREQ, "frequencies must be positive");
        fmin = std::min(fmin, f->f_hz[m]);
        fmax = std::max(fmax, f->f_hz[m]);
    }
    pl_design_info d{};
    d.lambda_min = PL_C0 / fmax;
    d.lambda_c = PL_C0 / (0.5 * (fmin + fmax));
    d.bandwidth = fmax - fmin;
    const double R = g->radius, L = g->chord_len;
    const double chord_angle = 2.0 * std::asin(L / (2.0 * R));
    d.theta_h_deg = g->n_sections * chord_angle * 180.0 / M_PI;
    const double scan_len = (s->n - 1) * s->dz;
    double theta_z = 2.0 * std::atan(scan_len / (2.0 * R));
    if (beamwidth_z_deg > 0) theta_z = std::min(theta_z, beamwidth_z_deg * M_PI / 180.0);
    d.theta_z_deg = theta_z * 180.0 / M_PI;
    const double R0 = R * std::cos(0.5 * chord_angle);       // chord to centre
    const double a = L + target_dim;
    d.max_rx_spacing = d.lambda_min * std::sqrt(0.25 * a * a + R0 * R0) / a;
    d.max_elem_spacing = g->mode == 0 ? 0.5 * d.max_rx_spacing : d.max_rx_spacing;
    d.max_scan_step = theta_z > 0 ? d.lambda_min / (4.0 * std::sin(0.5 * theta_z)) : HUGE_VAL;
    d.res_x = d.lambda_c / (4.0 * std::sin(0.5 * d.theta_h_deg * M_PI / 180.0));
    d.res_y = d.bandwidth > 0 ? PL_C0 / (2.0 * d.bandwidth) : HUGE_VAL;
    d.res_z = theta_z > 0 ? d.lambda_c / (4.0 * std::sin(0.5 * theta_z)) : HUGE_VAL;
    // actual spacing: largest gap between neighbouring elements of a section
    // (receive elements for the multistatic array: those used as receivers)
    double gap = 0.0;
    if (g->elem_xy && g->n_elem > 1) {
        for (int i = 0; i < g->n_elem; ++i) {
            bool rx = g->mode == 0;
            for (int p = 0; g->mode == 1 && p < g->n_pairs; ++p) rx = rx || g->pair_rx[p] == i;
            if (!rx) continue;
            double best = HUGE_VAL;
            for (int j = 0; j < g->n_elem; ++j) {
                if (j == i || (g->elem_section && g->elem_section[j] != g->elem_section[i])) continue;
                bool rj = g->mode == 0;
                for (int p = 0; g->mode == 1 && p < g->n_pairs; ++p) rj = rj || g->pair_rx[p] == j;
                if (!rj) continue;
                best = std::min(best, std::hypot(g->elem_xy[2 * i] - g->elem_xy[2 * j],
                                                 g->elem_xy[2 * i + 1] - g->elem_xy[2 * j + 1]));
            }
            if (best < HUGE_VAL) gap = std::max(gap, best);
        }
    }
    d.elem_spacing = gap;
    d.scan_step = s->dz;
    d.spacing_ok = gap <= d.max_elem_spacing ? 1 : 0;
    d.scan_step_ok = s->dz <= d.max_scan_step ? 1 : 0;
    *out = d;
    return PL_OK;
}
