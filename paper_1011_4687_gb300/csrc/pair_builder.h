// Host pair builder: environment input -> tiled Hermite distributions.
#pragma once

#include <cmath>
#include <string>
#include <vector>

#include "../../include/esp.h"
#include "esp_internal.h"

namespace esp {

struct HostEnv {
    std::vector<TileMeta> tiles;
    std::vector<float> rec32;      // FP32 distribution records
    std::vector<double> rec64;     // FP64 distribution records, then point records
    int64_t n_point_charges = 0;
    int64_t n_pairs_in = 0;
    int64_t n_distributions = 0;
    int64_t n_screened = 0;
    int64_t n_by_L[kMaxL + 1] = {0, 0, 0, 0, 0};
    int64_t n_near_tiles = 0;      // tiles eligible for the FP64 near path
    int tile_size = 64;
    // Grid of the FP32 high words of coordinates (a power of two): centres and
    // positions are split as x = hi + lo with hi a multiple of coord_quantum, so
    // P_hi - C_hi is exact in FP32 whenever |P_hi - C_hi| < 2^24 * coord_quantum.
    double coord_quantum = 1.0 / 1048576.0;
};

// hi word of x on the grid q (exact in double and in FP32 for |x| < 2^23 q)
inline double quantize_hi(double x, double q) { return std::nearbyint(x / q) * q; }

// Validate, fold, screen, sort and tile.  Returns ESP_OK or ESP_ERR_INVALID
// (with a message in err).
esp_status build_environment(const esp_point_charge *charges, int64_t n_charges,
                             const esp_gauss_pair *pairs, const double *weights, int64_t n_pairs,
                             const esp_options &opt, HostEnv &out, std::string &err);

// Boys tables for the FP32 and FP64 kernels (rows at T_i = i/8).
const std::vector<float> &boys_table32();
const std::vector<double> &boys_table64();

} // namespace esp
