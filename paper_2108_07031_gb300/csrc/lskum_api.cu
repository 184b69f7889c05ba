// C ABI of the solver (include/lskum.h): context life cycle, device memory,
// the pseudo-time iteration of Algorithm 1 as kernel launches (captured once
// into a CUDA graph and replayed), state transfer and diagnostics.

#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lskum_internal.h"
#include "lskum_kernels.cuh"

using namespace lskum;

namespace lskum {
namespace {
thread_local std::string g_last_error;
}
void set_last_error(const std::string& msg) { g_last_error = msg; }
static const char* last_error_cstr() { return g_last_error.c_str(); }
}  // namespace lskum

namespace {

constexpr int64_t kResCap = 1 << 20;
constexpr double kPi = 3.14159265358979323846;

struct Timer {
    std::vector<cudaEvent_t> ev;  // pairs
    double total_ms = 0.0;
    int64_t launches = 0;
};

}  // namespace

struct lskum_ctx {
    lskum_options opt{};
    int device = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    int block = kDefaultBlock;     // flux / update kernel
    int block_ls = kDefaultBlock;  // q-derivative kernels

    HostLayout host;
    bool mixed = false;
    DevGeom g{};
    DevGeom32 g32{};
    Physics ph{};
    DevState st{};
    std::vector<void*> allocations;

    V4* staging = nullptr;  // C x n x 4 in caller order (state transfer)
    V8* staging8 = nullptr; // C x n x 8 in caller order (derivative output)
    int* h_status = nullptr;             // pinned
    double* h_small = nullptr;           // pinned scratch for small reads

    bool have_state = false;
    int C = 1;                       // conditions solved together
    std::vector<double> mach, alpha; // free stream per condition
    V4* w_cond = nullptr;            // device copy of the free streams
    int64_t iters_done = 0;  // iterations since the last state reset

    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    bool use_graph = true;

    bool profiling = false;
    Timer timers[kNumKernelClasses];
    int64_t last_launches = 0;
};

namespace {

int fail(int code, const std::string& msg) {
    set_last_error(msg);
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(LSKUM_ERR_CUDA, m);
}

#define LSKUM_CUDA(call)                                        \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);     \
    } while (0)

template <typename T>
cudaError_t dev_alloc(lskum_ctx* c, T** p, size_t count) {
    void* raw = nullptr;
    cudaError_t e = cudaMalloc(&raw, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) c->allocations.push_back(raw);
    *p = static_cast<T*>(raw);
    return e;
}

template <typename T>
cudaError_t upload(lskum_ctx* c, const T** dst, const std::vector<T>& src) {
    T* p = nullptr;
    cudaError_t e = dev_alloc(c, &p, src.size());
    if (e != cudaSuccess) return e;
    if (!src.empty()) e = cudaMemcpy(p, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
    *dst = p;
    return e;
}

void release(lskum_ctx* c) {
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    for (auto& t : c->timers)
        for (auto e : t.ev) cudaEventDestroy(e);
    for (void* p : c->allocations) cudaFree(p);
    if (c->h_status) cudaFreeHost(c->h_status);
    if (c->h_small) cudaFreeHost(c->h_small);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
}

// Kernel launch wrapper that records CUDA events around a launch while
// profiling is on (one event pair per launch; resolved in lskum_kernel_time).
template <typename F>
cudaError_t timed(lskum_ctx* c, int cls, F&& launch) {
    if (!c->profiling) return launch();
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, c->stream);
    cudaError_t e = launch();
    cudaEventRecord(b, c->stream);
    c->timers[cls].ev.push_back(a);
    c->timers[cls].ev.push_back(b);
    return e;
}

int n_blocks(const lskum_ctx* c) { return int((c->g.n + c->block - 1) / c->block); }

// q-derivatives of the q buffer `qb` into dq[final] (FP64) or dq32[final]
// (mixed); returns the index of the buffer holding the result.
cudaError_t run_q_derivatives(lskum_ctx* c, int qb, int* final_buf, int64_t* launches) {
    cudaError_t e = timed(c, kLsFirst, [&] {
        return c->mixed ? launch_ls_first_mx(c->g, c->g32, c->st.qhl[qb], c->st.dq32[0], c->block_ls, c->stream)
                        : launch_ls_first(c->g, c->st.q[qb], c->st.dq[0], c->block_ls, c->stream);
    });
    if (e != cudaSuccess) return e;
    ++*launches;
    // buffer 0 holds the first-order result, used by every sweep; the
    // sweeps alternate between buffers 1 and 2
    int cur = 0;
    for (int it = 0; it < c->opt.inner_iters; ++it) {
        const int next = cur == 1 ? 2 : 1;
        e = timed(c, kLsInner, [&] {
            return c->mixed ? launch_ls_inner_mx(c->g, c->g32, c->st.dq32[0], c->st.dq32[cur],
                                                 c->st.dq32[next], c->block_ls, c->stream)
                            : launch_ls_inner(c->g, c->st.dq[0], c->st.dq[cur], c->st.dq[next],
                                              c->block_ls, c->stream);
        });
        if (e != cudaSuccess) return e;
        ++*launches;
        cur = next;
    }
    *final_buf = cur;
    return cudaSuccess;
}

cudaError_t launch_flux_any(lskum_ctx* c, int mode, int qb, int dbuf, int qout) {
    if (c->mixed)
        return launch_flux_mx(mode, c->g, c->g32, c->ph, c->st, c->st.qhl[qb], c->st.dq32[dbuf],
                              qout >= 0 ? c->st.qhl[qout] : nullptr, c->block, c->stream);
    if (c->opt.flux_split)
        return launch_flux_split(mode, c->g, c->ph, c->st, c->st.q[qb], c->st.dq[dbuf],
                                 qout >= 0 ? c->st.q[qout] : nullptr, c->block, c->stream);
    return launch_flux(mode, c->g, c->ph, c->st, c->st.q[qb], c->st.dq[dbuf],
                       qout >= 0 ? c->st.q[qout] : nullptr, c->block, c->stream);
}

// One pseudo-time iteration (Algorithm 1): four stages of q-derivatives and
// fused flux/update, then the residue. Starts and ends with q in st.q[0].
cudaError_t run_iteration(lskum_ctx* c, int64_t* launches) {
    int qcur = 0;
    for (int stage = 1; stage <= 4; ++stage) {
        int dbuf = 0;
        cudaError_t e = run_q_derivatives(c, qcur, &dbuf, launches);
        if (e != cudaSuccess) return e;
        e = timed(c, kFlux, [&] { return launch_flux_any(c, stage, qcur, dbuf, 1 - qcur); });
        if (e != cudaSuccess) return e;
        *launches += c->opt.flux_split ? 5 : 1;
        qcur = 1 - qcur;
        if (stage == 1) {
            e = timed(c, kReduce, [&] {
                return c->C == 1 ? launch_residue(c->st, n_blocks(c), c->g.n, c->stream)
                                 : launch_residue_cond(c->g, c->st, c->stream);
            });
            if (e != cudaSuccess) return e;
            *launches += c->C == 1 ? 1 : 2;
        }
    }
    return cudaSuccess;
}

cudaError_t refresh_mixed_q(lskum_ctx* c);

// After U changed from the host side: the mixed path's float-pair q.
cudaError_t refresh_mixed_q(lskum_ctx* c) {
    if (!c->mixed) return cudaSuccess;
    return launch_q_from_U_mx(c->g, c->ph, c->st.U, c->st.qhl[0], c->stream);
}

int reset_history(lskum_ctx* c) {
    LSKUM_CUDA(cudaMemsetAsync(c->st.iter_counter, 0, sizeof(unsigned long long), c->stream));
    LSKUM_CUDA(cudaMemsetAsync(c->st.status, 0, sizeof(int), c->stream));
    c->iters_done = 0;
    return LSKUM_OK;
}

int read_status(lskum_ctx* c, int* status) {
    LSKUM_CUDA(cudaMemcpyAsync(c->h_status, c->st.status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    LSKUM_CUDA(cudaStreamSynchronize(c->stream));
    *status = *c->h_status;
    return LSKUM_OK;
}

// Residues of iteration `iter` (0-based since the last reset), one per
// condition, into out[C].
int read_residue(lskum_ctx* c, int64_t iter, double* out) {
    const int64_t slot = iter % (kResCap / c->C);
    LSKUM_CUDA(cudaMemcpyAsync(c->h_small, c->st.res_hist + slot * c->C, sizeof(double) * c->C,
                               cudaMemcpyDeviceToHost, c->stream));
    LSKUM_CUDA(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < c->C; ++k) out[k] = c->h_small[k];
    return LSKUM_OK;
}

}  // namespace

extern "C" {

int lskum_default_options(lskum_options* o) {
    if (!o) return fail(LSKUM_ERR_INVALID_ARG, "null options");
    o->gamma = 1.4;
    o->cfl = 0.2;
    o->inner_iters = 2;
    o->order = 2;
    o->wall_factor = 2.0;
    o->outer_mode = LSKUM_OUTER_FREESTREAM;
    o->precision = LSKUM_FP64;
    o->reorder = 1;
    o->block_size = 0;
    o->check_every = 50;
    o->n_conditions = 1;
    o->flux_split = 0;
    o->weight_power = 0.0;
    return LSKUM_OK;
}

int lskum_create(int64_t n, const double* xy, const double* normals, const int8_t* flags,
                 const int32_t* nbr_offsets, const int32_t* nbr_idx, const lskum_options* opt,
                 lskum_ctx** out) {
    if (!out) return fail(LSKUM_ERR_INVALID_ARG, "null output pointer");
    *out = nullptr;
    lskum_options o;
    lskum_default_options(&o);
    if (opt) o = *opt;
    if (!(o.gamma > 1.0 && o.gamma < 2.0) || !(o.cfl > 0.0) || o.inner_iters < 0 ||
        o.inner_iters > 64 || (o.order != 1 && o.order != 2) || !(o.wall_factor > 0.0) ||
        (o.outer_mode != 0 && o.outer_mode != 1) ||
        (o.precision != LSKUM_FP64 && o.precision != LSKUM_MIXED) ||
        (o.block_size != 0 && o.block_size != 128 && o.block_size != 256) || o.check_every < 1 ||
        o.n_conditions < 1 || o.n_conditions > 256 || (o.n_conditions & (o.n_conditions - 1)) ||
        (o.flux_split != 0 && o.flux_split != 1) || (o.flux_split && o.precision != LSKUM_FP64) ||
        !(o.weight_power >= 0.0 && o.weight_power <= 8.0))
        return fail(LSKUM_ERR_INVALID_ARG, "invalid option value");

    lskum_ctx* c = new (std::nothrow) lskum_ctx();
    if (!c) return fail(LSKUM_ERR_INVALID_ARG, "out of host memory");
    c->opt = o;
    c->block = o.block_size ? o.block_size : kDefaultBlock;
    c->block_ls = c->block;
    c->mixed = o.precision == LSKUM_MIXED;
    c->C = o.n_conditions;
    c->mach.assign(c->C, 0.0);
    c->alpha.assign(c->C, 0.0);

    // host validation and layout first: input errors are reported without a GPU
    std::string err;
    int rc = build_layout(n, xy, normals, flags, nbr_offsets, nbr_idx, o, c->host, err);
    if (rc != LSKUM_OK) {
        delete c;
        return fail(rc, err);
    }
    int ndev = 0;
    cudaError_t ce = cudaGetDeviceCount(&ndev);
    if (ce != cudaSuccess || ndev == 0) {
        delete c;
        return fail(LSKUM_ERR_CUDA, std::string("no usable CUDA device: ") +
                                        (ce != cudaSuccess ? cudaGetErrorString(ce) : "none found"));
    }
    cudaGetDevice(&c->device);
    auto bail = [&](cudaError_t e, const char* where) {
        release(c);
        delete c;
        return cuda_fail(e, where);
    };
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(e, "cudaStreamCreate");
    c->stream = c->own_stream;

    const HostLayout& L = c->host;
    DevGeom& g = c->g;
    g.n = L.n;
    g.stride = L.stride;
    g.slots = L.slots;
    g.n_wall = int64_t(L.wall_id.size());
    g.cshift = 0;
    while ((1 << g.cshift) < c->C) ++g.cshift;
    g.cmask = uint32_t(c->C - 1);
    std::vector<double2> nrm2(L.n), nds2(L.wall_id.size());
    for (int64_t i = 0; i < L.n; ++i) nrm2[i] = make_double2(L.nrm[2 * i], L.nrm[2 * i + 1]);
    for (size_t k = 0; k < L.wall_id.size(); ++k) nds2[k] = make_double2(L.wall_nds[2 * k], L.wall_nds[2 * k + 1]);
    if ((e = upload(c, &g.cnt, L.cnt)) != cudaSuccess ||
        (e = upload(c, &g.flag, L.flag)) != cudaSuccess ||
        (e = upload(c, &g.nrm, nrm2)) != cudaSuccess ||
        (e = upload(c, &g.dmin, L.dmin)) != cudaSuccess ||
        (e = upload(c, &g.nbr, L.nbr)) != cudaSuccess ||
        (e = upload(c, &g.dev_to_user, L.dev_to_user)) != cudaSuccess ||
        (e = upload(c, &g.user_to_dev, L.user_to_dev)) != cudaSuccess ||
        (e = upload(c, &g.wall_id, L.wall_id)) != cudaSuccess ||
        (e = upload(c, &g.wall_nds, nds2)) != cudaSuccess)
        return bail(e, "upload of the cloud layout");

    if (!c->mixed) {
        if ((e = upload(c, &g.hdx, L.hdx)) != cudaSuccess ||
            (e = upload(c, &g.hdy, L.hdy)) != cudaSuccess ||
            (e = upload(c, &g.wx, L.wx)) != cudaSuccess ||
            (e = upload(c, &g.wy, L.wy)) != cudaSuccess ||
            (e = upload(c, &g.ws, L.ws)) != cudaSuccess ||
            (e = upload(c, &g.wn, L.wn)) != cudaSuccess)
            return bail(e, "upload of the FP64 cloud layout");
        std::vector<V4> lcoef(L.lc.size() / 4), lsum(L.lsum.size() / 4);
        std::memcpy(lcoef.data(), L.lc.data(), L.lc.size() * sizeof(double));
        std::memcpy(lsum.data(), L.lsum.data(), L.lsum.size() * sizeof(double));
        if ((e = upload(c, &g.lcoef, lcoef)) != cudaSuccess ||
            (e = upload(c, &g.lsum, lsum)) != cudaSuccess)
            return bail(e, "upload of the FP64 inner-sweep coefficients");
    } else {
        // FP32 records per neighbour entry: {ws, wn, hdx, hdy} and {wx, wy};
        // per point the coordinates as float pairs (device order)
        std::vector<float4> fxw(L.wx.size());
        std::vector<float2> lw2(L.wx.size());
        for (size_t i = 0; i < fxw.size(); ++i) {
            fxw[i] = make_float4(float(L.ws[i]), float(L.wn[i]), float(L.hdx[i]), float(L.hdy[i]));
            lw2[i] = make_float2(float(L.wx[i]), float(L.wy[i]));
        }
        std::vector<float4> xyhl(size_t(L.n));
        for (int64_t d = 0; d < L.n; ++d) {
            const double x = xy[2 * size_t(L.dev_to_user[d])], y = xy[2 * size_t(L.dev_to_user[d]) + 1];
            const float xh = float(x), yh = float(y);
            xyhl[size_t(d)] = make_float4(xh, yh, float(x - double(xh)), float(y - double(yh)));
        }
        if ((e = upload(c, &c->g32.fxw, fxw)) != cudaSuccess ||
            (e = upload(c, &c->g32.lw2, lw2)) != cudaSuccess ||
            (e = upload(c, &c->g32.xyhl, xyhl)) != cudaSuccess)
            return bail(e, "upload of the FP32 cloud layout");
    }

    DevState& st = c->st;
    const size_t N = size_t(L.n) * size_t(c->C);  // (point, condition) pairs
    const int nb = int((L.n + 127) / 128) + 1;  // block partials when C == 1
    if (c->mixed) {
        if ((e = dev_alloc(c, &st.qhl[0], N)) != cudaSuccess ||
            (e = dev_alloc(c, &st.qhl[1], N)) != cudaSuccess ||
            (e = dev_alloc(c, &st.dq32[0], N)) != cudaSuccess ||
            (e = dev_alloc(c, &st.dq32[1], N)) != cudaSuccess ||
            (e = dev_alloc(c, &st.dq32[2], N)) != cudaSuccess)
            return bail(e, "mixed-precision state allocation");
    } else {
        if ((e = dev_alloc(c, &st.q[1], N)) != cudaSuccess ||
            (e = dev_alloc(c, &st.dq[0], N)) != cudaSuccess ||
            (e = dev_alloc(c, &st.dq[1], N)) != cudaSuccess ||
            (e = dev_alloc(c, &st.dq[2], N)) != cudaSuccess)
            return bail(e, "FP64 state allocation");
    }
    if ((e = dev_alloc(c, &st.U, N)) != cudaSuccess || (e = dev_alloc(c, &st.U0, N)) != cudaSuccess ||
        (e = dev_alloc(c, &st.q[0], N)) != cudaSuccess ||
        (e = dev_alloc(c, &st.dt, N)) != cudaSuccess || (e = dev_alloc(c, &st.R, N)) != cudaSuccess ||
        (e = dev_alloc(c, &st.partials, size_t(nb))) != cudaSuccess ||
        (e = dev_alloc(c, &st.res_hist, size_t(kResCap))) != cudaSuccess ||
        (e = dev_alloc(c, &st.iter_counter, 1)) != cudaSuccess ||
        (e = dev_alloc(c, &st.status, 1)) != cudaSuccess ||
        (e = dev_alloc(c, &st.force_out, size_t(2 * c->C))) != cudaSuccess ||
        (e = dev_alloc(c, &c->w_cond, size_t(c->C))) != cudaSuccess ||
        (e = dev_alloc(c, &c->staging, N)) != cudaSuccess)
        return bail(e, "device state allocation");
    if (c->C > 1 &&
        ((e = dev_alloc(c, &st.r2, N)) != cudaSuccess ||
         (e = dev_alloc(c, &st.cpartials, size_t(kCondReduceBlocks) * c->C)) != cudaSuccess))
        return bail(e, "per-condition residue scratch");
    st.res_cap = kResCap;
    if ((e = cudaMallocHost(&c->h_status, sizeof(int) * 4)) != cudaSuccess ||
        (e = cudaMallocHost(&c->h_small, sizeof(double) * size_t(std::max(4, 2 * c->C)))) != cudaSuccess)
        return bail(e, "pinned host allocation");

    Physics& ph = c->ph;
    ph.gamma = o.gamma;
    ph.gm1 = o.gamma - 1.0;
    ph.gm1_inv = 1.0 / (o.gamma - 1.0);
    ph.cfl = o.cfl;
    ph.p_inf = 1.0 / o.gamma;
    ph.order = o.order;
    ph.outer_fixed = o.outer_mode == LSKUM_OUTER_FREESTREAM ? 1 : 0;

    if ((e = cudaMemsetAsync(st.iter_counter, 0, sizeof(unsigned long long), c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(st.status, 0, sizeof(int), c->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
        return bail(e, "initialisation");
    *out = c;
    return LSKUM_OK;
}

void lskum_destroy(lskum_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    release(c);
    delete c;
}

int lskum_set_stream(lskum_ctx* c, void* stream) {
    if (!c) return fail(LSKUM_ERR_INVALID_ARG, "null context");
    LSKUM_CUDA(cudaStreamSynchronize(c->stream));
    c->stream = stream ? static_cast<cudaStream_t>(stream) : c->own_stream;
    return LSKUM_OK;
}

int lskum_set_conditions(lskum_ctx* c, int n_cond, const double* mach, const double* alpha_deg) {
    if (!c || !mach || !alpha_deg) return fail(LSKUM_ERR_INVALID_ARG, "null argument");
    if (n_cond != c->C)
        return fail(LSKUM_ERR_INVALID_ARG, "n_cond = " + std::to_string(n_cond) +
                                               " differs from the context's n_conditions = " +
                                               std::to_string(c->C));
    std::vector<V4> W(c->C);
    for (int k = 0; k < c->C; ++k) {
        if (!(mach[k] >= 0.0) || !std::isfinite(mach[k]) || !std::isfinite(alpha_deg[k]))
            return fail(LSKUM_ERR_INVALID_ARG, "invalid free stream");
        const double a = alpha_deg[k] * kPi / 180.0;
        W[k] = V4{1.0, mach[k] * std::cos(a), mach[k] * std::sin(a), 1.0 / c->opt.gamma};
    }
    LSKUM_CUDA(cudaMemcpyAsync(c->w_cond, W.data(), sizeof(V4) * W.size(), cudaMemcpyHostToDevice,
                               c->stream));
    LSKUM_CUDA(launch_set_uniform(c->g, c->ph, c->w_cond, c->st.U, c->st.q[0], c->stream));
    LSKUM_CUDA(refresh_mixed_q(c));
    int rc = reset_history(c);
    if (rc != LSKUM_OK) return rc;
    LSKUM_CUDA(cudaStreamSynchronize(c->stream));  // W is a pageable host buffer
    c->mach.assign(mach, mach + c->C);
    c->alpha.assign(alpha_deg, alpha_deg + c->C);
    c->have_state = true;
    return LSKUM_OK;
}

int lskum_set_freestream(lskum_ctx* c, double mach, double alpha_deg) {
    if (!c) return fail(LSKUM_ERR_INVALID_ARG, "null context");
    std::vector<double> m(c->C, mach), a(c->C, alpha_deg);
    return lskum_set_conditions(c, c->C, m.data(), a.data());
}

int lskum_set_state(lskum_ctx* c, const double* prim) {
    if (!c || !prim) return fail(LSKUM_ERR_INVALID_ARG, "null argument");
    LSKUM_CUDA(cudaMemcpyAsync(c->staging, prim, sizeof(V4) * size_t(c->g.n) * c->C,
                               cudaMemcpyHostToDevice, c->stream));
    int rc = reset_history(c);
    if (rc != LSKUM_OK) return rc;
    LSKUM_CUDA(launch_set_prim(c->g, c->ph, c->staging, c->st.U, c->st.q[0], c->st.status, c->stream));
    LSKUM_CUDA(refresh_mixed_q(c));
    int status = 0;
    rc = read_status(c, &status);
    if (rc != LSKUM_OK) return rc;
    if (status) {
        reset_history(c);
        c->have_state = false;
        return fail(LSKUM_ERR_DIVERGED, "state has a non-finite value or rho <= 0 or p <= 0");
    }
    c->have_state = true;
    return LSKUM_OK;
}

int lskum_get_state(lskum_ctx* c, double* prim) {
    if (!c || !prim) return fail(LSKUM_ERR_INVALID_ARG, "null argument");
    if (!c->have_state) return fail(LSKUM_ERR_STATE, "no state set");
    LSKUM_CUDA(launch_get_prim(c->g, c->ph, c->st.U, c->staging, c->stream));
    LSKUM_CUDA(cudaMemcpyAsync(prim, c->staging, sizeof(V4) * size_t(c->g.n) * c->C,
                               cudaMemcpyDeviceToHost, c->stream));
    LSKUM_CUDA(cudaStreamSynchronize(c->stream));
    return LSKUM_OK;
}

int lskum_step(lskum_ctx* c, int n_iters) {
    if (!c || n_iters < 0) return fail(LSKUM_ERR_INVALID_ARG, "invalid argument");
    if (!c->have_state) return fail(LSKUM_ERR_STATE, "no state set");
    int64_t launches = 0;
    const bool graph = c->use_graph && !c->profiling;
    if (graph && !c->graph_exec && n_iters > 0) {
        int64_t cap_launches = 0;
        LSKUM_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = run_iteration(c, &cap_launches);
        cudaGraph_t gr = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(c->stream, &gr);
        if (e != cudaSuccess) return cuda_fail(e, "iteration capture");
        if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
        c->graph = gr;
        LSKUM_CUDA(cudaGraphInstantiate(&c->graph_exec, c->graph, 0));
    }
    for (int it = 0; it < n_iters; ++it) {
        if (graph) {
            LSKUM_CUDA(cudaGraphLaunch(c->graph_exec, c->stream));
            launches += 4 * (1 + c->opt.inner_iters + (c->opt.flux_split ? 5 : 1)) + (c->C == 1 ? 1 : 2);
        } else {
            cudaError_t e = run_iteration(c, &launches);
            if (e != cudaSuccess) return cuda_fail(e, "iteration launch");
        }
    }
    c->iters_done += n_iters;
    c->last_launches = launches;
    int status = 0;
    int rc = read_status(c, &status);
    if (rc != LSKUM_OK) return rc;
    if (status) return fail(LSKUM_ERR_DIVERGED, "non-finite or non-physical state during iteration");
    return LSKUM_OK;
}

int lskum_solve(lskum_ctx* c, int max_iters, double tol, int* iters_done) {
    if (!c || max_iters < 0 || !(tol > 0.0)) return fail(LSKUM_ERR_INVALID_ARG, "invalid argument");
    if (iters_done) *iters_done = 0;
    int done = 0;
    const int C = c->C;
    std::vector<double> first(C, 0.0), r(C, 0.0);
    int64_t scan_from = c->iters_done;
    while (done < max_iters) {
        const int chunk = std::min(c->opt.check_every, max_iters - done);
        int rc = lskum_step(c, chunk);
        done += chunk;
        if (iters_done) *iters_done = done;
        if (rc != LSKUM_OK) return rc;
        // first non-zero residue of this run, per condition
        for (int64_t k = scan_from; k < c->iters_done; ++k) {
            bool all = true;
            for (int m = 0; m < C; ++m) all = all && first[m] > 0.0;
            if (all) break;
            rc = read_residue(c, k, r.data());
            if (rc != LSKUM_OK) return rc;
            for (int m = 0; m < C; ++m)
                if (first[m] == 0.0 && r[m] > 0.0) first[m] = r[m];
        }
        scan_from = c->iters_done;
        rc = read_residue(c, c->iters_done - 1, r.data());
        if (rc != LSKUM_OK) return rc;
        bool converged = true;
        for (int m = 0; m < C; ++m) converged = converged && first[m] > 0.0 && r[m] <= tol * first[m];
        if (converged) break;
    }
    return LSKUM_OK;
}

int lskum_residual_norm(lskum_ctx* c, double* out) {
    if (!c || !out) return fail(LSKUM_ERR_INVALID_ARG, "null argument");
    if (c->iters_done == 0) {
        for (int k = 0; k < c->C; ++k) out[k] = 0.0;
        return LSKUM_OK;
    }
    return read_residue(c, c->iters_done - 1, out);
}

int lskum_forces(lskum_ctx* c, double* cl, double* cd) {
    if (!c || !cl || !cd) return fail(LSKUM_ERR_INVALID_ARG, "null argument");
    if (!c->have_state) return fail(LSKUM_ERR_STATE, "no state set");
    LSKUM_CUDA(launch_forces(c->g, c->ph, c->st, c->stream));
    LSKUM_CUDA(cudaMemcpyAsync(c->h_small, c->st.force_out, 2 * sizeof(double) * c->C,
                               cudaMemcpyDeviceToHost, c->stream));
    LSKUM_CUDA(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < c->C; ++k) {
        const double fx = c->h_small[2 * k], fy = c->h_small[2 * k + 1];
        const double a = c->alpha[k] * kPi / 180.0;
        const double qinf = 0.5 * c->mach[k] * c->mach[k];
        if (!(qinf > 0.0)) return fail(LSKUM_ERR_STATE, "forces need a free stream with M > 0");
        cl[k] = (-fx * std::sin(a) + fy * std::cos(a)) / qinf;
        cd[k] = (fx * std::cos(a) + fy * std::sin(a)) / qinf;
    }
    return LSKUM_OK;
}

int lskum_eval_residual(lskum_ctx* c, double* R) {
    if (!c || !R) return fail(LSKUM_ERR_INVALID_ARG, "null argument");
    if (!c->have_state) return fail(LSKUM_ERR_STATE, "no state set");
    int dbuf = 0;
    int64_t launches = 0;
    cudaError_t e = run_q_derivatives(c, 0, &dbuf, &launches);
    if (e != cudaSuccess) return cuda_fail(e, "q-derivatives");
    LSKUM_CUDA(launch_flux_any(c, 0, 0, dbuf, -1));
    LSKUM_CUDA(launch_gather_v4(c->g, c->st.R, c->staging, c->stream));
    LSKUM_CUDA(cudaMemcpyAsync(R, c->staging, sizeof(V4) * size_t(c->g.n) * c->C,
                               cudaMemcpyDeviceToHost, c->stream));
    LSKUM_CUDA(cudaStreamSynchronize(c->stream));
    return LSKUM_OK;
}

int lskum_eval_q_derivatives(lskum_ctx* c, double* qx, double* qy) {
    if (!c || !qx || !qy) return fail(LSKUM_ERR_INVALID_ARG, "null argument");
    if (!c->have_state) return fail(LSKUM_ERR_STATE, "no state set");
    if (!c->staging8) {
        LSKUM_CUDA(dev_alloc(c, &c->staging8, size_t(c->g.n) * c->C));
    }
    int dbuf = 0;
    int64_t launches = 0;
    cudaError_t e = run_q_derivatives(c, 0, &dbuf, &launches);
    if (e != cudaSuccess) return cuda_fail(e, "q-derivatives");
    if (c->mixed) {
        LSKUM_CUDA(launch_dq_to_user_mx(c->g, c->st.dq32[dbuf], c->staging8, c->stream));
    } else {
        LSKUM_CUDA(launch_gather_v8(c->g, c->st.dq[dbuf], c->staging8, c->stream));
    }
    std::vector<V8> h(size_t(c->g.n) * c->C);
    LSKUM_CUDA(cudaMemcpyAsync(h.data(), c->staging8, sizeof(V8) * h.size(), cudaMemcpyDeviceToHost, c->stream));
    LSKUM_CUDA(cudaStreamSynchronize(c->stream));
    for (size_t i = 0; i < h.size(); ++i)
        for (int m = 0; m < 4; ++m) {
            qx[4 * i + m] = h[i].x[m];
            qy[4 * i + m] = h[i].y[m];
        }
    return LSKUM_OK;
}

int lskum_info(lskum_ctx* c, int64_t* n_points, int64_t* n_wall, int* max_neighbours,
               int* n_conditions) {
    if (!c) return fail(LSKUM_ERR_INVALID_ARG, "null context");
    if (n_points) *n_points = c->g.n;
    if (n_wall) *n_wall = c->g.n_wall;
    if (max_neighbours) *max_neighbours = c->g.slots;
    if (n_conditions) *n_conditions = c->C;
    return LSKUM_OK;
}

int lskum_autotune(lskum_ctx* c, int trial_iters, int* best_block) {
    if (!c || trial_iters < 1) return fail(LSKUM_ERR_INVALID_ARG, "invalid argument");
    if (!c->have_state) return fail(LSKUM_ERR_STATE, "no state set");
    // keep the state (U and its FP64 q-variables, which set_state may have
    // formed from the primitive state directly): every trial restarts from it
    V4* saved = nullptr;
    const size_t N = size_t(c->g.n) * c->C;
    LSKUM_CUDA(cudaMalloc(&saved, 2 * sizeof(V4) * N));
    LSKUM_CUDA(cudaMemcpyAsync(saved, c->st.U, sizeof(V4) * N, cudaMemcpyDeviceToDevice, c->stream));
    LSKUM_CUDA(cudaMemcpyAsync(saved + N, c->st.q[0], sizeof(V4) * N, cudaMemcpyDeviceToDevice,
                               c->stream));
    const int candidates[2] = {128, 256};
    double best_ms = 1e300;
    int best = c->block, best_ls = c->block_ls;
    cudaEvent_t e0, e1;
    LSKUM_CUDA(cudaEventCreate(&e0));
    LSKUM_CUDA(cudaEventCreate(&e1));
    const bool was_profiling = c->profiling;
    c->profiling = false;
    for (int cand : candidates) {
        for (int cand_ls : candidates) {
            c->block = cand;
            c->block_ls = cand_ls;
            int64_t launches = 0;
            cudaError_t e = run_iteration(c, &launches);  // warm-up of this shape
            if (e != cudaSuccess) return cuda_fail(e, "autotune warm-up");
            LSKUM_CUDA(cudaEventRecord(e0, c->stream));
            for (int k = 0; k < trial_iters; ++k) {
                e = run_iteration(c, &launches);
                if (e != cudaSuccess) return cuda_fail(e, "autotune trial");
            }
            LSKUM_CUDA(cudaEventRecord(e1, c->stream));
            LSKUM_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            LSKUM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best_ms) {
                best_ms = ms;
                best = cand;
                best_ls = cand_ls;
            }
            LSKUM_CUDA(cudaMemcpyAsync(c->st.U, saved, sizeof(V4) * N, cudaMemcpyDeviceToDevice,
                                       c->stream));
            LSKUM_CUDA(cudaMemcpyAsync(c->st.q[0], saved + N, sizeof(V4) * N,
                                       cudaMemcpyDeviceToDevice, c->stream));
        }
    }
    c->profiling = was_profiling;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    LSKUM_CUDA(cudaStreamSynchronize(c->stream));
    cudaFree(saved);
    c->block = best;
    c->block_ls = best_ls;
    // the state is back to where it was: rebuild the mixed path's q (from U,
    // as set_state does), drop the captured graph (its launch shapes belong to
    // the old block size) and the trial history
    LSKUM_CUDA(refresh_mixed_q(c));
    if (c->graph_exec) {
        cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = nullptr;
    }
    if (c->graph) {
        cudaGraphDestroy(c->graph);
        c->graph = nullptr;
    }
    int rc = reset_history(c);
    if (rc != LSKUM_OK) return rc;
    LSKUM_CUDA(cudaStreamSynchronize(c->stream));
    if (best_block) *best_block = best * 1000 + best_ls;
    return LSKUM_OK;
}

static int resolve_timers(lskum_ctx* c) {
    LSKUM_CUDA(cudaStreamSynchronize(c->stream));
    for (auto& t : c->timers) {
        for (size_t k = 0; k + 1 < t.ev.size(); k += 2) {
            float ms = 0.f;
            LSKUM_CUDA(cudaEventElapsedTime(&ms, t.ev[k], t.ev[k + 1]));
            t.total_ms += ms;
            t.launches += 1;
            cudaEventDestroy(t.ev[k]);
            cudaEventDestroy(t.ev[k + 1]);
        }
        t.ev.clear();
    }
    return LSKUM_OK;
}

int lskum_profile(lskum_ctx* c, int enable) {
    if (!c) return fail(LSKUM_ERR_INVALID_ARG, "null context");
    int rc = resolve_timers(c);
    if (rc != LSKUM_OK) return rc;
    if (enable) {
        for (auto& t : c->timers) {
            t.total_ms = 0.0;
            t.launches = 0;
        }
    }
    c->profiling = enable != 0;
    return LSKUM_OK;
}

int lskum_kernel_time(lskum_ctx* c, int kernel, double* total_ms, int64_t* launches) {
    if (!c || kernel < 0 || kernel >= kNumKernelClasses)
        return fail(LSKUM_ERR_INVALID_ARG, "invalid argument");
    int rc = resolve_timers(c);
    if (rc != LSKUM_OK) return rc;
    if (total_ms) *total_ms = c->timers[kernel].total_ms;
    if (launches) *launches = c->timers[kernel].launches;
    return LSKUM_OK;
}

int64_t lskum_last_launch_count(lskum_ctx* c) { return c ? c->last_launches : -1; }

const char* lskum_error_string(int code) {
    switch (code) {
        case LSKUM_OK: return "ok";
        case LSKUM_ERR_INVALID_ARG: return "invalid argument";
        case LSKUM_ERR_BAD_CONNECTIVITY: return "bad connectivity";
        case LSKUM_ERR_DEGENERATE_STENCIL: return "degenerate stencil";
        case LSKUM_ERR_CUDA: return "CUDA error";
        case LSKUM_ERR_DIVERGED: return "diverged";
        case LSKUM_ERR_TIMEOUT: return "timeout";
        case LSKUM_ERR_STATE: return "call out of order";
        default: return "unknown error";
    }
}

const char* lskum_last_error(void) { return lskum::last_error_cstr(); }

}  // extern "C"
