// Device-side launch interface of the potential kernels.
#pragma once

#include <cuda_runtime.h>

#include "esp_internal.h"

namespace esp {

// Recentred positions, structure of arrays: FP64 copy and FP32 hi + lo split,
// hi on the environment's coordinate grid and lo = fp32(x - hi), so FP32 code
// forms P - C as (P_hi - C_hi) + (P_lo - C_lo) with an exact first difference.
struct Staged {
    double *x64, *y64, *z64;
    float *xh, *yh, *zh, *xl, *yl, *zl;
};

// FP32C tile groups: FP64 point charges, FP32 point charges, then one group
// per L (long- and short-range tiles of that L together).
constexpr int kMaxTileGroups = 7;

struct EvalArgs {
    int n_pos;
    int n_splits;     // tiles are dealt round-robin to this many splits
    int n_tiles;
    int tile_size;
    Staged pos;
    const TileMeta *tiles;
    const float *rec32;
    const double *rec64;
    const float *boys32;
    const double *boys64;
    double *partial;  // [n_splits][n_pos], FP64
    float near_r;     // FP32C: FP64 re-evaluation radius around a tile's bounding sphere
    // FP32C deal by tile group: group g holds tiles [grp_tile[g], grp_tile[g+1])
    // and takes the splits [grp_split[g], grp_split[g+1]) (grp_split[n_groups] =
    // n_splits), so each CTA runs the code of one class.  One group over all
    // tiles is the plain round-robin deal.
    int n_groups;
    int grp_tile[kMaxTileGroups + 1];
    int grp_split[kMaxTileGroups + 1];
};

// the plain deal: every tile in one group over n_splits splits
ESP_HD void single_group(EvalArgs &a)
{
    a.n_groups = 1;
    a.grp_tile[0] = 0;
    a.grp_tile[1] = a.n_tiles;
    a.grp_split[0] = 0;
    a.grp_split[1] = a.n_splits;
}

// One system of a batched evaluation (device-side table entry).
struct SysDesc {
    const TileMeta *tiles;
    const float *rec32;
    const double *rec64;
    const double *pos_in; // [n_pos][3] device
    double *V_out;        // [n_pos] device
    double *partial;      // [splits][n_pos]
    Staged st;
    double qm[3];
    double quantum;
    int n_tiles, tile_size, n_pos, splits, blocks, item_begin, pos_begin;
    float near_r;
    int sorted;           // stage in spatial order (slot_of / perm below are [n_pos] scratch)
    int *slot_of, *perm;
};

struct BatchHeader {
    int n_sys, n_items, n_pos_total, pad;
};

// Batched pipeline on stream s: staging, persistent potential kernel over all
// (system, block, split) items, reduction into each system's V_out.  The
// counter must be zero when the potential kernel starts.
// max_sys: the number of systems (one spatial-order CTA each, for systems marked sorted)
cudaError_t launch_batch(int precision, const BatchHeader *hdr, const SysDesc *sys, int max_sys, int *counter,
                         int max_items,
                         const float *boys32, const double *boys64, int tile_cap, int threads, int ppt,
                         int num_sms, int max_pos_total, cudaStream_t s);
bool batch_shape_supported(int precision, int threads, int ppt);

// slot_of (optional, from launch_sort): the staged slot of each input position
cudaError_t launch_stage(const double *pos_in, int n, const double center[3], double quantum, const Staged &st,
                         cudaStream_t s, const int *slot_of = nullptr);
// Spatial order of n positions (stable counting sort by the Morton code of a
// 16^3 cell grid over [-8, 8]^3 bohr about center).  scratch holds
// sort_scratch_ints(n) ints; on return *slot_of[i] is the slot of position i
// and *perm[slot] its input index (both inside scratch).
constexpr int kSortSide = 16;
constexpr int kSortCells = kSortSide * kSortSide * kSortSide;
constexpr int kSortThreads = 256;
constexpr double kSortHalf = 8.0;
constexpr int kSortMinPositions = 4096; // fewer: the order is not worth its three launches
size_t sort_scratch_ints(int n);
cudaError_t launch_sort(const double *pos_in, int n, const double center[3], int *scratch, int **slot_of, int **perm,
                        cudaStream_t s);
// precision: 0 = FP64, 1 = FP32C.  threads in {64, 128, 256}, ppt in {1, 2, 4}.
cudaError_t launch_potential(int precision, const EvalArgs &a, int threads, int ppt, cudaStream_t s);
size_t potential_smem_bytes(int precision, int tile_size);
// Launch shapes compiled into the library: FP64 threads {64,128,256} x ppt {1,2};
// FP32C (64,{2,4}), (128,{1,2,4}), (256,{1,2}).
bool potential_shape_supported(int precision, int threads, int ppt);
// Few positions per call (n <= kSmallN): environment entries spread over the
// threads of n_splits CTAs per chunk of kSmallChunk positions (grid n_splits x
// chunks), partial[split][n], then one CTA per position sums the partials
// into V in a fixed order.  Entries are evaluated in FP64, except the FP32
// point charges (class kClassPoint32) when fp32 is set: those take the
// compensated FP32 form of the main kernel (hi/lo offsets, symmetric rsqrt,
// low word of the charge), sum per thread in FP32 and reduce across the CTA
// as (sum, compensation) pairs before the FP64 partial.
constexpr int kSmallN = 128;
constexpr int kSmallChunk = 16;      // positions of one CTA, held in registers
constexpr int kSmallNDistributions = 16; // calls above this many positions take the
                                         // few-position path only for environments of point charges
struct SmallArgs {
    int n_pos;
    int n_tiles;
    const double *pos_in;  // [n_pos][3] device positions (recentred inside the kernel)
    double cx, cy, cz;     // QM centre
    const TileMeta *tiles;
    const double *rec64;
    const float *rec32;
    const double *boys64;
    double quantum;        // coordinate grid of the FP32 hi words
    int fp32;              // FP32 point charges in compensated FP32
    int64_t p32_off;       // float offset of the FP32 point records (contiguous, n_p32 of them)
    int n_p32;
    double *partial;
};
int small_n_splits(int n_tiles, int num_sms, int n);
cudaError_t launch_small_n(const SmallArgs &a, int n_splits, double *V, cudaStream_t s);
// perm (optional, from launch_sort): V[perm[slot]] receives the sum of slot
cudaError_t launch_reduce(const double *partial, int n_splits, int n, double *V, cudaStream_t s,
                          const int *perm = nullptr);
cudaError_t launch_walkers(const double *V, int n_walkers, int n_elec, double *E, cudaStream_t s);

} // namespace esp
