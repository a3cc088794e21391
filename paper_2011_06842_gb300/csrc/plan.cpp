// Host-side planning of the FEWHA operator (Ramlau & Stadler, Sec. 2-4).
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <complex>

namespace fewha {

using cplx = std::complex<double>;

// ---------------------------------------------------------------------------
// Daubechies taps (Sec. 3: periodic orthonormal Daubechies wavelets)
//
// |H(w)|^2 = 2 cos^{2N}(w/2) P_N(sin^2(w/2)), P_N(y) = sum_{k<N} C(N-1+k,k) y^k.
// The roots of P_N are found with the Weierstrass (Durand-Kerner) iteration
// followed by Newton polishing; each root y maps to the pair of z with
// y = (2 - z - 1/z)/4 and the one inside the unit circle is kept.
// h(z) = c (1 + z^{-1})^N prod (1 - z_k z^{-1}), scaled to sum h = sqrt(2).
// ---------------------------------------------------------------------------
static double binom(int n, int k)
{
    double r = 1.0;
    for (int i = 1; i <= k; i++) r = r * (n - k + i) / i;
    return r;
}

static cplx poly_eval(const std::vector<double> &c, cplx x)  // c[0] + c[1] x + ...
{
    cplx v = 0.0;
    for (int i = (int)c.size() - 1; i >= 0; i--) v = v * x + c[i];
    return v;
}

bool daubechies_taps(int N, std::vector<double> &h)
{
    if (N < 1 || 2 * N > kMaxTaps) return false;
    std::vector<double> pc(N);
    for (int k = 0; k < N; k++) pc[k] = binom(N - 1 + k, k);
    int deg = N - 1;
    std::vector<cplx> roots(deg);
    if (deg > 0) {
        // monic version for Durand-Kerner
        std::vector<double> mc(pc.size());
        for (size_t i = 0; i < pc.size(); i++) mc[i] = pc[i] / pc[deg];
        const cplx seed(0.4, 0.9);
        for (int i = 0; i < deg; i++) roots[i] = std::pow(seed, i);
        for (int it = 0; it < 500; it++) {
            double change = 0.0;
            for (int i = 0; i < deg; i++) {
                cplx den = 1.0;
                for (int j = 0; j < deg; j++)
                    if (j != i) den *= roots[i] - roots[j];
                cplx d = poly_eval(mc, roots[i]) / den;
                roots[i] -= d;
                change = std::max(change, std::abs(d));
            }
            if (change < 1e-15) break;
        }
        std::vector<double> dc(deg);  // derivative coefficients
        for (int i = 1; i <= deg; i++) dc[i - 1] = i * pc[i];
        for (auto &r : roots)
            for (int it = 0; it < 4; it++) {
                cplx d = poly_eval(dc, r);
                if (std::abs(d) == 0.0) break;
                r -= poly_eval(pc, r) / d;
            }
    }
    std::vector<cplx> poly{1.0};
    auto mul = [&](cplx a0, cplx a1) {  // poly *= (a0 + a1 z^{-1})
        std::vector<cplx> out(poly.size() + 1, 0.0);
        for (size_t i = 0; i < poly.size(); i++) {
            out[i] += a0 * poly[i];
            out[i + 1] += a1 * poly[i];
        }
        poly.swap(out);
    };
    for (const cplx &y : roots) {
        cplx a = 1.0 - 2.0 * y;
        cplx disc = std::sqrt(a * a - 1.0);
        cplx z = (std::abs(a + disc) < 1.0) ? a + disc : a - disc;
        mul(1.0, -z);
    }
    for (int i = 0; i < N; i++) mul(1.0, 1.0);
    h.assign(poly.size(), 0.0);
    double s = 0.0;
    for (size_t i = 0; i < poly.size(); i++) {
        h[i] = poly[i].real();
        s += h[i];
    }
    for (auto &v : h) v *= std::sqrt(2.0) / s;
    return true;
}

// ---------------------------------------------------------------------------
// Geometry (Sec. 2; layer domain reading: every projected pupil node lies at
// least one cell inside the layer grid, max |coordinate| / d_l = n_l/2 - 2,
// node k at (k - n_l/2) d_l)
// ---------------------------------------------------------------------------
static double cone(const fewha_gs &g, double h) { return g.H > 0 ? 1.0 - h / g.H : 1.0; }

// Band class of coefficient (r, q) of an n x n Mallat layout with J levels:
// 0 = approximation, then 1 + 3 (s-1) + (quad-1) for detail level s = 1..J
// (coarse to fine) and quadrant 1 (low y, high x), 2 (high y, low x), 3 (high-high).
static int band_class(int n, int J, int r, int q, int *level)
{
    int a = n >> J;
    if (r < a && q < a) {
        *level = 0;
        return 0;
    }
    int half = a;
    for (int s = 1; s <= J; s++, half *= 2) {
        if (r < 2 * half && q < 2 * half) {
            int quad = (r < half) ? 1 : ((q < half) ? 2 : 3);
            *level = s;
            return 1 + 3 * (s - 1) + (quad - 1);
        }
    }
    *level = -1;
    return -1;
}

int build_plan(const fewha_geometry &g, Plan &p)
{
    if (g.n_sub < 1 || g.n_gs < 1 || g.n_gs > FEWHA_MAX_GS || g.n_layers < 1 ||
        g.n_layers > FEWHA_MAX_LAYERS || !(g.D > 0) || g.obstruction < 0 || g.obstruction >= 1 ||
        !(g.r0 > 0) || !(g.alpha >= 0) || g.wavelet_N < 1 || 2 * g.wavelet_N > kMaxTaps ||
        g.precision < FEWHA_F64 || g.precision > FEWHA_BF16S)
        return FEWHA_ERR_ARG;
    if (g.tile != 0 && g.tile != 8 && g.tile != 16 && g.tile != 32) return FEWHA_ERR_ARG;
    p.geom = g;
    p.G = g.n_gs;
    p.L = g.n_layers;
    p.ns = g.n_sub;
    p.m = g.n_sub + 1;
    p.ds = g.D / g.n_sub;
    if (p.m > 4096) return FEWHA_ERR_ARG;
    if (!daubechies_taps(g.wavelet_N, p.taps)) return FEWHA_ERR_ARG;
    for (int k = 0; k < p.G; k++) {
        const fewha_gs &s = g.gs[k];
        if (!std::isfinite(s.theta_x) || !std::isfinite(s.theta_y) || !(s.weight >= 0) || s.n_sub < 0 ||
            s.n_sub > 4095)
            return FEWHA_ERR_ARG;
    }

    // sensors: sizes and block offsets
    p.gns.resize(p.G);
    p.gm.resize(p.G);
    p.tab_off.resize(p.G);
    p.psi_off.assign(p.G + 1, 0);
    p.slope_off.assign(p.G + 1, 0);
    p.mask_off.assign(p.G + 1, 0);
    p.m_max = 0;
    long tab_total = 0;
    for (int k = 0; k < p.G; k++) {
        const int ns = g.gs[k].n_sub > 0 ? g.gs[k].n_sub : g.n_sub;
        p.gns[k] = ns;
        p.gm[k] = ns + 1;
        p.m_max = std::max(p.m_max, ns + 1);
        p.tab_off[k] = tab_total;
        tab_total += 2L * g.n_layers * (ns + 1);
        p.psi_off[k + 1] = p.psi_off[k] + (long)(ns + 1) * (ns + 1);
        p.slope_off[k + 1] = p.slope_off[k] + 2L * ns * ns;
        p.mask_off[k + 1] = p.mask_off[k] + (long)ns * ns;
    }

    // lit subapertures: centre radius within [obstruction D/2, D/2]; the
    // single subaperture of a 1x1 sensor sees the whole pupil (always lit)
    p.mask.assign((size_t)p.mask_off[p.G], 0);
    double rin = 0.5 * g.obstruction * g.D, rout = 0.5 * g.D;
    for (int k = 0; k < p.G; k++) {
        const int ns = p.gns[k];
        const double dsg = g.D / ns;
        for (int i = 0; i < ns; i++)
            for (int j = 0; j < ns; j++) {
                double cx = -0.5 * g.D + (j + 0.5) * dsg, cy = -0.5 * g.D + (i + 0.5) * dsg;
                double r = std::sqrt(cx * cx + cy * cy);
                p.mask[(size_t)p.mask_off[k] + (size_t)i * ns + j] = (ns == 1 || (r >= rin && r <= rout)) ? 1 : 0;
            }
    }

    // layer grids
    p.lay_d.resize(p.L);
    p.lay_off.resize(p.L + 1);
    p.n = 0;
    for (int l = 0; l < p.L; l++) {
        const fewha_layer &ly = g.layers[l];
        int n = ly.n;
        if (n < 8 || n > FEWHA_MAX_GRID || (n & (n - 1)) || ly.J < 1 || (n >> ly.J) < 1 ||
            !(ly.cn2 > 0) || ly.delta == 0 || !std::isfinite(ly.delta) || ly.h < 0)
            return FEWHA_ERR_GEOMETRY;
        double R = 0.0;
        for (int k = 0; k < p.G; k++) {
            const fewha_gs &s = g.gs[k];
            if (s.H > 0 && ly.h >= s.H) return FEWHA_ERR_GEOMETRY;
            double tx = std::fabs(s.theta_x * ly.h), ty = std::fabs(s.theta_y * ly.h);
            R = std::max(R, cone(s, ly.h) * 0.5 * g.D + std::max(tx, ty));
        }
        p.lay_d[l] = R / (0.5 * n - 2.0);
        p.lay_off[l] = p.n;
        p.n += (long)n * n;
    }
    p.lay_off[p.L] = p.n;

    // interpolation tables of P_g and the ranges of P_g^T
    size_t nt = (size_t)p.G * p.L * 2;
    p.fk.assign((size_t)tab_total, 0);
    p.fw.assign((size_t)tab_total, 0.0);
    p.alo.assign(nt * FEWHA_MAX_GRID, 0);
    p.ahi.assign(nt * FEWHA_MAX_GRID, 0);
    for (int k = 0; k < p.G; k++) {
        const fewha_gs &s = g.gs[k];
        for (int l = 0; l < p.L; l++) {
            const fewha_layer &ly = g.layers[l];
            double sc = cone(s, ly.h), d = p.lay_d[l];
            for (int ax = 0; ax < 2; ax++) {
                size_t base = ((size_t)k * p.L + l) * 2 + ax;  // P_g^T ranges
                const size_t tb = p.tab(k, l, ax);             // P_g tables of this sensor
                const int mg = p.gm[k];
                const double dsg = g.D / p.gns[k];
                double shift = (ax == 0 ? s.theta_x : s.theta_y) * ly.h;
                for (int j = 0; j < mg; j++) {
                    double x = -0.5 * g.D + j * dsg;
                    double f = (sc * x + shift) / d + 0.5 * ly.n;
                    int kk = (int)std::floor(f);
                    if (kk < 0 || kk + 1 > ly.n - 1) return FEWHA_ERR_GEOMETRY;
                    p.fk[tb + j] = kk;
                    double w = f - kk;
                    if (g.precision == FEWHA_BF16S) {  // weights stored in bfloat16
                        float wf = (float)w;
                        unsigned int u;
                        std::memcpy(&u, &wf, 4);
                        u += 0x7FFFu + ((u >> 16) & 1u);
                        u &= 0xFFFF0000u;
                        std::memcpy(&wf, &u, 4);
                        w = wf;
                    }
                    p.fw[tb + j] = w;
                }
                for (int node = 0; node < ly.n; node++) {
                    int lo = mg, hi = 0;
                    for (int j = 0; j < mg; j++) {
                        int kk = p.fk[tb + j];
                        if (kk == node || kk + 1 == node) {
                            lo = std::min(lo, j);
                            hi = std::max(hi, j + 1);
                        }
                    }
                    if (lo >= hi) lo = hi = 0;
                    p.alo[base * FEWHA_MAX_GRID + node] = lo;
                    p.ahi[base * FEWHA_MAX_GRID + node] = hi;
                }
            }
        }
    }

    // fitting step of Algorithm 3 (reading: one DM conjugated to the ground,
    // actuators on the pupil nodes): on-axis projection, no cone, no shift
    p.fit_k.assign((size_t)p.L * p.m, 0);
    p.fit_w.assign((size_t)p.L * p.m, 0.0);
    p.fit_ok = 1;
    for (int l = 0; l < p.L; l++) {
        const int n = g.layers[l].n;
        for (int j = 0; j < p.m; j++) {
            const double f = (-0.5 * g.D + j * p.ds) / p.lay_d[l] + 0.5 * n;
            const int kk = (int)std::floor(f);
            if (kk < 0 || kk + 1 > n - 1) {
                p.fit_ok = 0;
                continue;
            }
            p.fit_k[(size_t)l * p.m + j] = kk;
            p.fit_w[(size_t)l * p.m + j] = f - kk;
        }
    }

    // prior D (reading: Kolmogorov spectrum in the wavelet domain)
    //   D = kappa_l 2^{(11/3) s}, kappa_l = 2^{-(11/3) J} / (0.5 * 6.88 (d_l/r0_l)^{5/3}),
    //   r0_l = r0 cn2_l^{-3/5}, s = 0 approximation, 1..J detail levels coarse to fine.
    p.alpha_d.assign(p.n, 0.0);
    p.coef_class.assign(p.n, 0);
    p.n_classes = 0;
    std::vector<int> class_base(p.L);
    for (int l = 0; l < p.L; l++) {
        const fewha_layer &ly = g.layers[l];
        class_base[l] = p.n_classes;
        p.n_classes += 1 + 3 * ly.J;
        double r0l = g.r0 * std::pow(ly.cn2, -0.6);
        double kappa = std::pow(2.0, -(11.0 / 3.0) * ly.J) /
                       (0.5 * 6.88 * std::pow(p.lay_d[l] / r0l, 5.0 / 3.0));
        for (int r = 0; r < ly.n; r++)
            for (int q = 0; q < ly.n; q++) {
                int lev;
                int cls = band_class(ly.n, ly.J, r, q, &lev);
                long i = p.lay_off[l] + (long)r * ly.n + q;
                p.alpha_d[i] = g.alpha * kappa * std::pow(2.0, (11.0 / 3.0) * lev);
                p.coef_class[i] = class_base[l] + cls;
            }
        // sampled coefficients of every band: offsets {nb/4, 3nb/4} per axis
        for (int s = 0; s <= ly.J; s++) {
            int nb = (ly.n >> ly.J) << (s > 0 ? s - 1 : 0);
            for (int quad = (s == 0 ? 0 : 1); quad <= (s == 0 ? 0 : 3); quad++) {
                int r0 = (quad == 2 || quad == 3) ? nb : 0;
                int q0 = (quad == 1 || quad == 3) ? nb : 0;
                int offs[2] = {nb / 4, (3 * nb) / 4};
                int no = offs[0] == offs[1] ? 1 : 2;
                int cls = class_base[l] + (s == 0 ? 0 : 1 + 3 * (s - 1) + (quad - 1));
                for (int a = 0; a < no; a++)
                    for (int b = 0; b < no; b++) {
                        p.sample_idx.push_back(p.lay_off[l] + (long)(r0 + offs[a]) * ly.n + (q0 + offs[b]));
                        p.sample_class.push_back(cls);
                    }
            }
        }
    }
    return FEWHA_OK;
}

}  // namespace fewha
