// Predicted Effective Bandwidth (Sec. 3.4.3, Eq. 2) for bandwidth-sensitive
// requests, evaluated once on the host in double precision.
//
// Eq. 2 is a regression over the link counts of an allocation -- x double
// NVLinks, y single NVLinks, z PCIe links -- with fourteen features: the
// counts, their inverse-linear terms 1/(c+1), the pairwise products, their
// inverses 1/(cc'+1), the triple product and its inverse 1/(xyz+1), weighted
// by the coefficients of Table 2.
//
// The device never evaluates Eq. 2.  A sensitive request is scored with
// per-class codes (4096 per double NVLink, 64 per single NVLink, 1 per PCIe
// link), so the integer score of a match is the index (x * 64 + y) * 64 + z of
// its link counts; the tables built here map that index to the dense rank of
// its predicted bandwidth (equal values share a rank) and to round(1000 *
// EffBW).  The fused tail takes the argmax over ranks, so the floating-point
// comparison that decides the winner is made once, here, in double.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <vector>

#include "mapa_internal.h"

namespace mapa {

namespace {

// Table 2 (theta_1 .. theta_14), in the order of the features below.
constexpr double kTheta[14] = {16.396, 4.536, 1.556,  -20.694, -9.467, 7.615,  -7.973,
                               12.733, -4.195, -8.413, 62.851,  27.418, -5.114, -46.973};

}  // namespace

double effbw_predict(int x, int y, int z) {
    const double X = x, Y = y, Z = z;
    const double feature[14] = {
        X,       Y,       Z,                                         // linear
        1.0 / (X + 1.0), 1.0 / (Y + 1.0), 1.0 / (Z + 1.0),          // inverse-linear
        X * Y,   Y * Z,   Z * X,                                     // pairwise
        1.0 / (X * Y + 1.0), 1.0 / (Y * Z + 1.0), 1.0 / (Z * X + 1.0),  // inverse-pairwise
        X * Y * Z, 1.0 / (X * Y * Z + 1.0),                          // triplet, inverse-triplet
    };
    double f = 0.0;
    for (int i = 0; i < 14; ++i) f += kTheta[i] * feature[i];
    return f;
}

int32_t effbw_class_code(int32_t weight) {
    if (weight == 50) return kEffbwRadix * kEffbwRadix;  // double NVLink-v2
    if (weight == 25 || weight == 20) return kEffbwRadix;  // single NVLink v2 / v1
    if (weight == 12) return 1;                          // PCIe
    return 0;
}

void effbw_tables(std::vector<int32_t> *rank, std::vector<int32_t> *milli) {
    constexpr int R = kEffbwRadix;
    const int n = R * R * R;
    std::vector<double> f(static_cast<size_t>(n));
    for (int x = 0; x < R; ++x)
        for (int y = 0; y < R; ++y)
            for (int z = 0; z < R; ++z) f[static_cast<size_t>((x * R + y) * R + z)] = effbw_predict(x, y, z);
    std::vector<int32_t> order(static_cast<size_t>(n));
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return f[a] < f[b]; });
    rank->assign(static_cast<size_t>(n), 0);
    milli->assign(static_cast<size_t>(n), 0);
    int32_t r = 0;
    for (int i = 0; i < n; ++i) {
        if (i > 0 && f[order[i]] != f[order[i - 1]]) ++r;
        (*rank)[order[i]] = r;
    }
    for (int i = 0; i < n; ++i) (*milli)[i] = static_cast<int32_t>(std::llround(1000.0 * f[i]));
}

}  // namespace mapa

extern "C" int mapa_effbw_predict(int32_t x, int32_t y, int32_t z, double *out) {
    if (!out) return MAPA_E_INVALID;
    if (x < 0 || y < 0 || z < 0 || x >= mapa::kEffbwRadix || y >= mapa::kEffbwRadix || z >= mapa::kEffbwRadix)
        return MAPA_E_RANGE;
    *out = mapa::effbw_predict(x, y, z);
    return MAPA_OK;
}
