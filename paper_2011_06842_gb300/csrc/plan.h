// Host-side planning of the FEWHA operator: geometry, interpolation tables,
// Daubechies taps, prior and the preconditioner's sampling plan.
// Internal header of libfewha (not part of the C ABI).
#pragma once
#include <vector>

#include "../../include/fewha.h"

namespace fewha {

constexpr int kMaxTaps = 8;

struct Plan {
    fewha_geometry geom;
    int G = 0, L = 0, ns = 0, m = 0;  // guide stars, layers, subapertures across, pupil nodes across
    long n = 0;                       // unknowns
    double ds = 0;                    // subaperture size of the geometry's grid (the mirror's)
    std::vector<double> taps;         // Daubechies low-pass h_0..h_{2N-1}
    // sensors: per guide star g its subapertures across (gns), pupil nodes
    // across (gm = gns + 1) and offsets of its blocks: P_g tables (tab_off,
    // 2 L gm entries), adjoint wavefront (psi_off, gm^2), slopes (slope_off,
    // 2 gns^2), mask (mask_off, gns^2); the last three with a G-th entry (the
    // total); m_max = largest gm
    std::vector<int> gns, gm;
    std::vector<long> tab_off, psi_off, slope_off, mask_off;
    int m_max = 0;
    size_t tab(int g, int l, int axis) const { return tab_off[g] + ((size_t)l * 2 + axis) * gm[g]; }
    std::vector<unsigned char> mask;  // lit subapertures, sensor after sensor
    std::vector<double> lay_d;        // layer grid spacing
    std::vector<long> lay_off;        // L+1 offsets into the coefficient vector
    // P_g tables, index tab(g, l, axis) + j  (axis 0 = x, 1 = y; j < gm[g])
    std::vector<int> fk;              // lower node index of pupil node j on layer l
    std::vector<double> fw;           // fractional position in that cell
    // P_g^T ranges, index ((g*L + l)*2 + axis)*FEWHA_MAX_GRID + k: pupil nodes
    // [alo, ahi) whose cell touches layer node k
    std::vector<int> alo, ahi;
    // fitting onto the ground DM (actuators on the pupil nodes), on-axis: per
    // (layer l, pupil index j) the lower node and fractional position, both axes
    std::vector<int> fit_k;
    std::vector<double> fit_w;
    int fit_ok = 0;                   // every actuator projects inside every layer grid
    std::vector<double> alpha_d;      // n, alpha * D
    // preconditioner sampling: class of every coefficient, and the sampled
    // coefficients (global index, class)
    int n_classes = 0;
    std::vector<int> coef_class;
    std::vector<long> sample_idx;
    std::vector<int> sample_class;
};

// Daubechies-N low-pass taps from the spectral factorisation of the
// half-band polynomial (own complex root finder).  Returns false on failure.
bool daubechies_taps(int N, std::vector<double> &h);

// Validates the geometry and fills every host table.  Returns FEWHA_OK or
// FEWHA_ERR_ARG / FEWHA_ERR_GEOMETRY.
int build_plan(const fewha_geometry &g, Plan &p);

}  // namespace fewha
