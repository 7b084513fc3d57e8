// Host pair builder: environment input -> tiled Hermite distributions.
#pragma once

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
    int tile_size = 128;
};

// Validate, fold, screen, sort and tile.  Returns ESP_OK or ESP_ERR_INVALID
// (with a message in err).
esp_status build_environment(const esp_point_charge *charges, int64_t n_charges,
                             const esp_gauss_pair *pairs, const double *weights, int64_t n_pairs,
                             const esp_options &opt, HostEnv &out, std::string &err);

// Boys tables for the FP32 and FP64 kernels (rows at T_i = i/8).
const std::vector<float> &boys_table32();
const std::vector<double> &boys_table64();

} // namespace esp
