// diag_tc_plan.h -- host plan of the tensor-core variance kernel (diag_tc.cu)
// and the packed-tile numbering it shares with the packing kernel.
#pragma once
#include <cstdint>
#include <vector>

#include "analysis.h"

#ifdef __CUDACC__
#define SPI_HD __host__ __device__
#else
#define SPI_HD
#endif

namespace spi {

constexpr int kDiagTcMinPivots = 32;  // default of spi_options.diag_tc_min_pivots
constexpr int kDiagTcMaxBlock = 128;  // right-hand sides of a variance block the kernel takes
constexpr int kDiagTcRows = 128;      // rows of a packed tile (the MMA's M)
constexpr int kDiagTcK = 32;          // K columns of a packed tile

struct DiagTcHost {
    int32_t ntc = 0;              // supernodes on the tensor cores
    int64_t npt = 0;              // packed left-operand tiles (per band)
    int32_t ndt = 0;              // inverted 128 x 128 diagonal tiles (per band)
    std::vector<uint8_t> tc;      // [ns] 1 = on the tensor cores
    std::vector<int64_t> tptr;    // [ns] first packed tile of the supernode
    std::vector<int32_t> xptr;    // [ns] first diagonal tile of the supernode
    std::vector<int32_t> ptiles;  // [npt][4] (supernode, row tile, K chunk, 0)
    std::vector<int32_t> dtiles;  // [ndt][2] (supernode, own row tile)
};

// Packed tiles of a supernode with k pivots are numbered row tile by row tile:
// own row tile rt < T (T = ceil(k / 128)) has K chunks of 32 up to the end of its
// diagonal block, 4 (rt + 1) of them (all ceil(k / 32) for the last); each row
// tile below has all nch = ceil(k / 32).  First tile of row tile rt:
SPI_HD inline int64_t diag_tc_tile_offset(int32_t T, int32_t nch, int32_t rt) {
    return rt < T ? 2 * (int64_t)rt * (rt + 1) : 2 * (int64_t)(T - 1) * T + nch + (int64_t)(rt - T) * nch;
}
SPI_HD inline int32_t diag_tc_row_chunks(int32_t T, int32_t nch, int32_t rt) { return rt < T - 1 ? 4 * (rt + 1) : nch; }

void build_diag_tc(const Symbolic& S, int min_k, DiagTcHost& h);
// TF32 MMA flops (three products per output, padded tiles) of one pass over a plan
double diag_tc_mma_flops(const Symbolic& S, const DiagTcHost& h, const DiagPlan& dp);

}  // namespace spi
