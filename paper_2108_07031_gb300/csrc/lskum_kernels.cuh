// Device data layout and kernel launchers of the q-LSKUM solver.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace lskum {

// 4-vector per point (primitive, conserved or q-variables), 32-byte aligned
// so one record is one DRAM sector.
struct __align__(32) V4 {
    double a, b, c, d;
};

// q-derivatives of one point: (q_x[4], q_y[4]), 64-byte aligned.
struct __align__(64) V8 {
    double x[4];
    double y[4];
};

// Mixed precision: q as a pair of floats (hi + lo carries the FP64 value to
// ~2^-48, so differences of nearby q are exact to FP32 precision of the
// difference), and (q_x, q_y) in FP32.
struct __align__(32) QHL {
    float4 hi;
    float4 lo;
};
struct __align__(32) D8f {
    float4 x;
    float4 y;
};

// FP32 copies of the slot-major per-neighbour arrays (mixed precision).
struct DevGeom32 {
    // slot-major [slot][stride], one record per neighbour entry so a kernel
    // fetches its per-neighbour constants with one vector load
    const float4* fxw;  // {ws, wn, hdx, hdy}: split-stencil weights (Eq. 24), half offsets
    const float2* lw2;  // {wx, wy}: least-squares weights (Eq. 11), both q-derivative sweeps
    // per point (device order): the coordinates as float pairs {x hi, y hi,
    // x lo, y lo} (hi + lo = the FP64 coordinate to ~2^-48), so the inner
    // sweeps form the half offsets (P_j - P_i)/2 in FP32 to FP32 precision of
    // the offset itself, from a gathered 16-byte record, instead of streaming
    // them per neighbour entry
    const float4* xyhl;
};

// Static cloud data on the device (device point order).
struct DevGeom {
    int64_t n;
    int64_t stride;  // row length of the slot-major arrays
    int slots;
    // Conditions (free streams) solved together: C = 2^cshift, condition
    // innermost. State index t = (point << cshift) | condition; thread t
    // handles one (point, condition) pair, so the 32 lanes of a warp share one
    // point's connectivity and weights (one broadcast load) and gather the
    // neighbours' states of 32 consecutive conditions (one contiguous read).
    int cshift;
    uint32_t cmask;
    const int32_t* cnt;
    const int8_t* flag;
    const double2* nrm;
    const double* dmin;
    const uint32_t* nbr;  // [slot][stride] packed entries (lskum_internal.h)
    const double* hdx;
    const double* hdy;
    const double* wx;
    const double* wy;
    const double* ws;
    const double* wn;
    // FP64 inner sweeps: per slot {wx hdx, wx hdy, wy hdx, wy hdy}, per point
    // their sums over the stencil
    const V4* lcoef;
    const V4* lsum;
    const int32_t* dev_to_user;
    const int32_t* user_to_dev;
    int64_t n_wall;
    const int32_t* wall_id;
    const double2* wall_nds;
};

struct Physics {
    double gamma;
    double gm1;      // gamma - 1
    double gm1_inv;  // 1 / (gamma - 1)
    double cfl;
    double p_inf;
    int order;        // 1 or 2
    int outer_fixed;  // far-field points hold the free stream
};

// Mutable solver state (device order).
struct DevState {
    V4* U;     // conserved state
    V4* U0;    // state at the start of the iteration
    V4* q[2];  // q-variables, double-buffered across stages
    V8* dq[3]; // q-derivatives: [0] first order (kept for the FP64 inner sweeps),
               // [1], [2] alternate across inner iterations
    double* dt;
    QHL* qhl[2];  // mixed precision: q-variables as float pairs
    D8f* dq32[3]; // mixed precision: q-derivatives in FP32, [0] first order, [1], [2] sweeps
    V4* R;     // residual output of the evaluation mode
    double* partials;  // per-block partial sums (scratch)
    double* r2;        // C > 1: stage-1 R_rho^2 per (point, condition) (scratch)
    double* cpartials; // C > 1: per-(block, condition) partial sums (scratch)
    double* res_hist;  // residue per iteration (ring buffer)
    int64_t res_cap;
    unsigned long long* iter_counter;
    int* status;       // bit 0: non-physical state seen
    double* force_out; // (Fx, Fy)
};

constexpr int kDefaultBlock = 128;
constexpr int kReduceBlock = 512;
constexpr int kCondReduceBlocks = 304;  // phase-1 blocks of the per-condition residue

enum KernelClass { kFlux = 0, kLsFirst = 1, kLsInner = 2, kReduce = 3, kNumKernelClasses = 4 };

// State index of (point d, condition c).
__host__ __device__ __forceinline__ int64_t sidx(const DevGeom& g, int64_t d, uint32_t c) {
    return (d << g.cshift) | int64_t(c);
}

// Launchers (return cudaGetLastError()).
cudaError_t launch_ls_first(const DevGeom& g, const V4* q, V8* dq, int block, cudaStream_t s);
cudaError_t launch_ls_inner(const DevGeom& g, const V8* dq_first, const V8* dq_in, V8* dq_out, int block,
                            cudaStream_t s);
// mode 0: evaluate R only (written to st.R); mode 1..4: SSP-RK stage.
cudaError_t launch_flux(int mode, const DevGeom& g, const Physics& ph, const DevState& st,
                        const V4* q_in, const V8* dq, V4* q_out, int block, cudaStream_t s);
// The paper's four split-flux kernels + a stage kernel (ablation of launch_flux;
// 5 launches; uses st.R as the accumulator).
cudaError_t launch_flux_split(int mode, const DevGeom& g, const Physics& ph, const DevState& st,
                              const V4* q_in, const V8* dq, V4* q_out, int block, cudaStream_t s);
cudaError_t launch_residue(const DevState& st, int nblocks, int64_t n, cudaStream_t s);
// C > 1: residue per condition from st.r2 (two deterministic phases).
cudaError_t launch_residue_cond(const DevGeom& g, const DevState& st, cudaStream_t s);
// W_cond: device array of C primitive free-stream states.
cudaError_t launch_set_uniform(const DevGeom& g, const Physics& ph, const V4* W_cond, V4* U, V4* q,
                               cudaStream_t s);
cudaError_t launch_set_prim(const DevGeom& g, const Physics& ph, const V4* W_user, V4* U, V4* q,
                            int* status, cudaStream_t s);
cudaError_t launch_get_prim(const DevGeom& g, const Physics& ph, const V4* U, V4* W_user,
                            cudaStream_t s);
cudaError_t launch_q_from_U(const DevGeom& g, const Physics& ph, const V4* U, V4* q, cudaStream_t s);
cudaError_t launch_gather_v4(const DevGeom& g, const V4* src_dev, V4* dst_user, cudaStream_t s);
cudaError_t launch_gather_v8(const DevGeom& g, const V8* src_dev, V8* dst_user, cudaStream_t s);
cudaError_t launch_forces(const DevGeom& g, const Physics& ph, const DevState& st,
                          cudaStream_t s);

// Mixed-precision launchers (lskum_kernels_mixed.cu).
cudaError_t launch_ls_first_mx(const DevGeom& g, const DevGeom32& g32, const QHL* q, D8f* dq,
                               int block, cudaStream_t s);
cudaError_t launch_ls_inner_mx(const DevGeom& g, const DevGeom32& g32, const D8f* dq_first,
                               const D8f* dq_in, D8f* dq_out, int block, cudaStream_t s);
cudaError_t launch_flux_mx(int mode, const DevGeom& g, const DevGeom32& g32, const Physics& ph,
                           const DevState& st, const QHL* q_in, const D8f* dq, QHL* q_out,
                           int block, cudaStream_t s);
cudaError_t launch_q_from_U_mx(const DevGeom& g, const Physics& ph, const V4* U, QHL* q,
                               cudaStream_t s);
cudaError_t launch_dq_to_user_mx(const DevGeom& g, const D8f* src, V8* dst_user, cudaStream_t s);

}  // namespace lskum
