// Internal declarations shared by the host set-up (lskum_setup.cpp), the
// device kernels (lskum_kernels.cu) and the C ABI (lskum_api.cu).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/lskum.h"

namespace lskum {

// Neighbour entries of the device layout pack the neighbour's device index
// with the two split-stencil codes of Eq. 14:
//   bits 0..25  neighbour index (n <= 2^26)
//   bits 26..27 s-stencil: 0 none, 1 "+" (ds < 0, dGs+/ds), 2 "-" (ds > 0, dGs-/ds)
//   bits 28..29 n-stencil: 0 none, 1 "+" (dn < 0, dGn+/dn), 2 "-" (dn > 0, dGn-/dn)
constexpr int kIndexBits = 26;
constexpr uint32_t kIndexMask = (1u << kIndexBits) - 1u;
constexpr int kMaxPoints = 1 << kIndexBits;

// Host-side product of lskum_create's set-up, in device point order.
struct HostLayout {
    int64_t n = 0;
    int64_t stride = 0;  // slot-array row length (n rounded up to 32)
    int slots = 0;       // max neighbours of any point
    std::vector<int32_t> dev_to_user;  // device id -> caller id
    std::vector<int32_t> user_to_dev;  // caller id -> device id
    std::vector<int32_t> cnt;          // neighbours per point
    std::vector<int8_t> flag;
    std::vector<double> nrm;   // n x 2 normals (boundary points), (0, 1) interior
    std::vector<double> dmin;  // min neighbour distance
    // slot-major [slot][stride] arrays
    std::vector<uint32_t> nbr;  // packed entry (index | codes)
    std::vector<double> hdx, hdy;  // half of the global offsets x_j - x_i, y_j - y_i
    std::vector<double> wx, wy;    // full-stencil least-squares weights (Eq. 11)
    std::vector<double> ws, wn;    // split-stencil weights of d/ds and d/dn (Eq. 24)
    // FP64 inner sweeps (Eq. 29) split as q_x = (first-order q_x) - sum_j wx_j
    // (hdx_j (qx_j - qx_i) + hdy_j (qy_j - qy_i)), likewise q_y: per slot the
    // products {wx hdx, wx hdy, wy hdx, wy hdy} (4 per slot, [slot][stride]),
    // per point their sums over the stencil (4 per point). FP64 layouts only.
    std::vector<double> lc;
    std::vector<double> lsum;
    // wall loops for the force integral: device ids and n_i ds_i
    std::vector<int32_t> wall_id;
    std::vector<double> wall_nds;  // n_wall x 2
};

// Validates the caller's cloud and builds the device layout. Returns LSKUM_OK
// or an error code with a message in `err`.
int build_layout(int64_t n, const double* xy, const double* normals, const int8_t* flags,
                 const int32_t* offsets, const int32_t* idx, const lskum_options& opt,
                 HostLayout& out, std::string& err);

void set_last_error(const std::string& msg);

}  // namespace lskum
