// C ABI of libsgw: context management, host orchestration of the kernels, and the FP64
// host routines (gapped-filter coefficients, Bessel coefficients).  See include/sgw.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <initializer_list>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/sgw.h"
#include "sgw_internal.cuh"

using cd = std::complex<double>;

struct sgw_ctx {
    int n = 0;
    int64_t ng = 0;
    double h = 0, dV = 0, L = 0, ecut = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    int max_batch = 0;
    double emin = 0, emax = 0;
    bool have_spectrum = false;
    bool have_potential = false;
    // device memory owned by the context
    float2* tw = nullptr;      // [n] exp(-2 pi i m / n)
    float* vloc = nullptr;     // [ng]
    float2* W = nullptr;       // [max_batch][ng]
    float2* B1 = nullptr;      // [max_batch][ng]
    float2* B2 = nullptr;      // [max_batch][ng]
    sgw::VecInfo* info = nullptr;  // [max_batch]
    float2* kbc = nullptr;     // [max_batch][n_proj]
    float2* kbp = nullptr;     // [max_batch][total_slots][4] per-plane partial projections
    sgw::KBDev kb;
    double* scal = nullptr;    // small FP64 scratch
    // lazily grown work areas
    static constexpr int kWorkSlots = 11;
    void* work[kWorkSlots] = {nullptr};
    size_t work_sz[kWorkSlots] = {0};
    float2* twM = nullptr;
    int twM_n = 0;
    std::vector<sgw::VecInfo> info_host;
    // instrumentation: launch counter and CUDA-event timing per kernel kind
    int64_t launches = 0;
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending[SGW_PROF_KINDS];
    double prof_ms[SGW_PROF_KINDS] = {0};
    int64_t prof_n[SGW_PROF_KINDS] = {0};
    double prof_bytes[SGW_PROF_KINDS] = {0};   // algorithmic (compulsory) HBM bytes of the launches
    // CUDA graphs of whole propagation loops, keyed by the call's arguments and buffers
    bool graph_mode = false;
    struct GraphEntry {
        std::vector<uint64_t> key;
        cudaGraphExec_t exec;
        int64_t n_launch;
    };
    std::vector<GraphEntry> graphs;
    // split-operator KB factors: orthonormalised projectors per support point (atom-major, like
    // kb.sup_idx), atoms grouped by 3D colour, per-atom M_a = R E R^T (host, 4 x 4), and the
    // complex factors e^{-i tau M_a} - 1 for tau = +dt/2 and -dt/2 of the last dt
    float4* kbq = nullptr;
    int* acol_atoms = nullptr;
    std::vector<int> acol_off;
    std::vector<double> kb_m;
    // one device table per dt used so far (graphs keep pointing at the table of their dt)
    std::vector<std::pair<double, float2*>> split_tabs;
    // launch tuning hints (sgw_set_tuning / sgw_autotune); no result depends on them
    int tune[SGW_TUNE_KEYS] = {1, 0, 0, 0, 0};
    std::string err;
};

static std::string g_setup_err;

namespace sgw {
// Errors of calls that have no context are reported through sgw_last_error(NULL).
void set_global_error(const char* msg) { g_setup_err = msg; }
}  // namespace sgw

namespace {
cudaEvent_t ev_get(sgw_ctx* c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
// Bracket one kernel launch: counts it and, when profiling, records events around it on the
// context's stream.
struct Launch {
    sgw_ctx* c;
    int kind;
    cudaEvent_t a = nullptr;
    Launch(sgw_ctx* ctx_, int kind_, int n_kernels = 1, double bytes = 0.0) : c(ctx_), kind(kind_) {
        c->launches += n_kernels;
        if (c->prof) {
            c->prof_bytes[kind] += bytes;
            a = ev_get(c);
            cudaEventRecord(a, c->stream);
        }
    }
    ~Launch() {
        if (a) {
            cudaEvent_t b = ev_get(c);
            cudaEventRecord(b, c->stream);
            c->ev_pending[kind].push_back({a, b});
        }
    }
};
// Resolve pending event pairs into accumulated milliseconds (synchronises the stream).
void prof_flush(sgw_ctx* c) {
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    for (int k = 0; k < SGW_PROF_KINDS; ++k) {
        for (auto& pr : c->ev_pending[k]) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) {
                c->prof_ms[k] += ms;
                c->prof_n[k] += 1;
            }
            c->ev_pool.push_back(pr.first);
            c->ev_pool.push_back(pr.second);
        }
        c->ev_pending[k].clear();
    }
    cudaGetLastError();
}
}  // namespace

namespace {

sgw_status fail(sgw_ctx* c, sgw_status s, const std::string& msg) {
    if (c) c->err = msg;
    else g_setup_err = msg;
    return s;
}

// Device buffers the kernels read or write with 16-byte vector accesses or bulk copies.
bool misaligned(std::initializer_list<const void*> ps) {
    for (const void* p : ps)
        if (reinterpret_cast<uintptr_t>(p) & 15u) return true;
    return false;
}
#define SGW_ALIGNED(ctx, ...) \
    if (misaligned({__VA_ARGS__})) return fail(ctx, SGW_EINVAL, "device buffers must be 16-byte aligned")

#define CK(call)                                                                                      \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return fail(ctx, SGW_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));         \
    } while (0)

#define CKL()                                                                                         \
    do {                                                                                              \
        cudaError_t e_ = cudaGetLastError();                                                          \
        if (e_ != cudaSuccess) return fail(ctx, SGW_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
    } while (0)

void clear_graphs(sgw_ctx* ctx) {
    for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.exec);
    ctx->graphs.clear();
}

// Grow work area `slot` to at least `bytes`.
sgw_status work(sgw_ctx* ctx, int slot, size_t bytes, void** out) {
    if (ctx->work_sz[slot] < bytes) {
        clear_graphs(ctx);
        if (ctx->work[slot]) {
            cudaStreamSynchronize(ctx->stream);
            cudaFree(ctx->work[slot]);
            ctx->work[slot] = nullptr;
            ctx->work_sz[slot] = 0;
        }
        cudaError_t e = cudaMalloc(&ctx->work[slot], bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, SGW_ENOMEM, "work area allocation failed: " + std::to_string(bytes) + " bytes");
        }
        ctx->work_sz[slot] = bytes;
    }
    *out = ctx->work[slot];
    return SGW_OK;
}

std::vector<float2> twiddles(int n) {
    std::vector<float2> t(n);
    for (int m = 0; m < n; ++m) {
        const double a = -2.0 * M_PI * (double)m / (double)n;
        t[m] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    return t;
}

float2 f2(cd z) { return make_float2((float)z.real(), (float)z.imag()); }

// ---- Bessel J_k(a), k = 0..K, by Miller's backward recurrence normalised with
//      J_0 + 2 sum_{k>=1} J_{2k} = 1 (J.C.P. Miller's method as given by
//      Abramowitz & Stegun 9.12 / Numerical Recipes).
std::vector<double> bessel_j(int K, double a) {
    std::vector<double> J(K + 1, 0.0);
    if (std::fabs(a) < 1e-300) {
        J[0] = 1.0;
        return J;
    }
    const int start = 2 * ((std::max(K, (int)std::ceil(std::fabs(a))) + 30 + (int)std::sqrt(40.0 * (K + 30))) / 2);
    std::vector<double> j(start + 2, 0.0);
    j[start + 1] = 0.0;
    j[start] = 1e-30;
    for (int k = start; k >= 1; --k) {
        j[k - 1] = 2.0 * k / a * j[k] - j[k + 1];
        if (std::fabs(j[k - 1]) > 1e250) {  // rescale to avoid overflow
            for (int q = k - 1; q <= start + 1; ++q) j[q] *= 1e-250;
        }
    }
    double norm = j[0];
    for (int k = 2; k <= start; k += 2) norm += 2.0 * j[k];
    for (int k = 0; k <= K; ++k) J[k] = j[k] / norm;
    return J;
}

// Clenshaw step plan of a Chebyshev sum sum_{k=0}^{K} c_k T_k(H~) psi (optionally times a phase).
struct Step {
    cd cpsi[2], ch[2], c2[2];
    int b1;     // 0: psi, 1: X, 2: Y
    int b2;     // -1: none, 1: X, 2: Y
    int out;    // 1: X, 2: Y, 3: final output
};

// c[set][k]: coefficient sets (set 1 only used when two_sets).  ch multiplies 2 H~ b1.
std::vector<Step> clenshaw_plan(const std::vector<cd>* c, const cd* phase, int K) {
    std::vector<Step> plan;
    if (K == 0) return plan;
    if (K == 1) {  // S = c0 psi + c1 H~ psi
        Step s;
        for (int q = 0; q < 2; ++q) {
            s.cpsi[q] = phase[q] * c[q][0];
            s.ch[q] = phase[q] * c[q][1] * 0.5;
            s.c2[q] = 0;
        }
        s.b1 = 0; s.b2 = -1; s.out = 3;
        plan.push_back(s);
        return plan;
    }
    // first: b_{K-1} = c_{K-1} psi + 2 c_K H~ psi  -> X
    {
        Step s;
        for (int q = 0; q < 2; ++q) { s.cpsi[q] = c[q][K - 1]; s.ch[q] = c[q][K]; s.c2[q] = 0; }
        s.b1 = 0; s.b2 = -1; s.out = 1;
        plan.push_back(s);
    }
    if (K == 2) {  // S = (c0 - c2) psi + H~ b1
        Step s;
        for (int q = 0; q < 2; ++q) { s.cpsi[q] = phase[q] * (c[q][0] - c[q][2]); s.ch[q] = phase[q] * 0.5; s.c2[q] = 0; }
        s.b1 = 1; s.b2 = -1; s.out = 3;
        plan.push_back(s);
        return plan;
    }
    // second: b_{K-2} = (c_{K-2} - c_K) psi + 2 H~ b_{K-1}  -> Y
    {
        Step s;
        for (int q = 0; q < 2; ++q) { s.cpsi[q] = c[q][K - 2] - c[q][K]; s.ch[q] = 1.0; s.c2[q] = 0; }
        s.b1 = 1; s.b2 = -1; s.out = 2;
        plan.push_back(s);
    }
    // b_{k+1} lives in `last`, b_{k+2} in `prev`; b_k overwrites b_{k+2}
    int last = 2, prev = 1;
    for (int k = K - 3; k >= 1; --k) {
        Step s;
        for (int q = 0; q < 2; ++q) { s.cpsi[q] = c[q][k]; s.ch[q] = 1.0; s.c2[q] = -1.0; }
        s.b1 = last; s.b2 = prev; s.out = prev;
        plan.push_back(s);
        std::swap(last, prev);
    }
    Step s;
    for (int q = 0; q < 2; ++q) { s.cpsi[q] = phase[q] * c[q][0]; s.ch[q] = phase[q] * 0.5; s.c2[q] = -phase[q]; }
    s.b1 = last; s.b2 = prev; s.out = 3;
    plan.push_back(s);
    return plan;
}

// Free every KB device array of the context
void free_kb(sgw_ctx* ctx) {
    sgw::KBDev& kb = ctx->kb;
    void* ptrs[] = {kb.atom_nproj, kb.atom_off, kb.sup_idx, kb.sup_beta, kb.atom_e, kb.plane_off, kb.slot_atom,
                    kb.kbe_col, kb.kbe_os, kb.kbe_beta, kb.kbe_slot_beg, kb.kbe_slot_end, kb.atom_pos_off,
                    kb.atom_pos, ctx->kbc, ctx->kbp};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    kb = sgw::KBDev();
    ctx->kbc = nullptr;
    ctx->kbp = nullptr;
    void* sp[] = {ctx->kbq, ctx->acol_atoms};
    for (void* p : sp)
        if (p) cudaFree(p);
    for (auto& t : ctx->split_tabs) cudaFree(t.second);
    ctx->split_tabs.clear();
    ctx->kbq = nullptr;
    ctx->acol_atoms = nullptr;
    ctx->acol_off.clear();
    ctx->kb_m.clear();
}

// KB table pointers of a plane-step launch
void set_kb_args(const sgw_ctx* ctx, sgw::StepArgs& a) {
    const sgw::KBDev& kb = ctx->kb;
    a.plane_off = kb.plane_off;
    a.slot_atom = kb.slot_atom;
    a.kbe_col = kb.kbe_col;
    a.kbe_os = kb.kbe_os;
    a.kbe_beta = kb.kbe_beta;
    a.kbe_slot_beg = kb.kbe_slot_beg;
    a.kbe_slot_end = kb.kbe_slot_end;
    a.max_colors = kb.max_colors;
    a.max_plane_slots = kb.max_plane_slots;
    a.total_slots = kb.total_slots;
    a.n_proj = kb.n_proj;
}

// Run one Chebyshev sum over a batch.  psi_in: real-space input; out: result (may alias psi_in).
// W must hold the forward xy transform of psi_in on entry when w_ready; on exit it holds the
// transform of the output when want_wout.
sgw_status run_series(sgw_ctx* ctx, const std::vector<Step>& plan, const float2* psi_in, float2* out, int batch,
                      const float* vpot, const float* dvpot, const sgw::VecInfo* info, bool w_ready, bool want_wout,
                      int vrows = 1) {
    cudaStream_t st = ctx->stream;
    const int n = ctx->n;
    const float kscale = (float)std::pow(2.0 * M_PI / ctx->L, 2);
    const double ebar = 0.5 * (ctx->emax + ctx->emin), de = 0.5 * (ctx->emax - ctx->emin);
    if (plan.empty()) {
        if (out != psi_in) CK(cudaMemcpyAsync(out, psi_in, sizeof(float2) * ctx->ng * batch, cudaMemcpyDeviceToDevice, st));
        return SGW_OK;
    }
    if (!w_ready) {
        Launch L(ctx, SGW_PROF_PLANE_FWD, 1, 16.0 * (double)ctx->ng * batch);
        sgw::launch_plane_fwd(n, psi_in, ctx->W, batch, ctx->tw, st);
        CKL();
    }
    auto buf = [&](int id) -> float2* {
        return id == 0 ? const_cast<float2*>(psi_in) : (id == 1 ? ctx->B1 : (id == 2 ? ctx->B2 : out));
    };
    for (size_t i = 0; i < plan.size(); ++i) {
        const Step& s = plan[i];
        const float2* b1 = buf(s.b1);
        if (ctx->kb.n_atoms > 0) {
            if (i == 0 && !w_ready) {
                // gathered psi (8 B) per support point and vector, plus the support index and beta (20 B)
                Launch L(ctx, SGW_PROF_KB, 1, (double)ctx->kb.n_sup * (8.0 * batch + 20.0));
                sgw::launch_kb_project(n, ctx->kb, b1, batch, (float)ctx->dV, ctx->kbc, st);
            } else {
                // the previous plane pass left per-plane partial projections of b1
                Launch L(ctx, SGW_PROF_KB, 1, 32.0 * (double)ctx->kb.total_slots * batch);
                sgw::launch_kb_reduce(ctx->kb, ctx->kbp, batch, (float)ctx->dV, ctx->kbc, st);
            }
            CKL();
        }
        {
            Launch L(ctx, SGW_PROF_PENCIL, 1, 16.0 * (double)ctx->ng * batch);
            sgw::launch_pencil(n, ctx->W, batch, 0, kscale, (float)ctx->ecut, ctx->tw, st,
                               ctx->tune[SGW_TUNE_PENCIL_LOOKAHEAD], nullptr, 0.f, ctx->tune[SGW_TUNE_LINE_FORM]);
            CKL();
        }
        sgw::StepArgs a{};
        a.W = ctx->W;
        const bool last = (i + 1 == plan.size());
        a.Wout = (!last || want_wout) ? ctx->W : nullptr;
        a.b1 = b1;
        a.b2 = s.b2 >= 0 ? buf(s.b2) : nullptr;
        a.psi = psi_in;
        a.out = buf(s.out);
        a.vpot = vpot;
        a.dvpot = dvpot;
        a.info = info;
        a.kbc = ctx->kb.n_atoms > 0 ? ctx->kbc : nullptr;
        a.kbp = (ctx->kb.n_atoms > 0 && a.Wout != nullptr) ? ctx->kbp : nullptr;
        set_kb_args(ctx, a);
        a.total_slots = ctx->kb.total_slots;
        a.n_proj = ctx->kb.n_proj;
        a.ebar = (float)ebar;
        a.alpha = (float)(2.0 / de);
        a.pf_ahead = ctx->tune[SGW_TUNE_PLANE_LOOKAHEAD];
        a.pf_operands = ctx->tune[SGW_TUNE_PLANE_OPERANDS];
        for (int q = 0; q < 2; ++q) {
            a.coef.cpsi[q] = f2(s.cpsi[q]);
            a.coef.ch[q] = f2(s.ch[q]);
            a.coef.c2[q] = f2(s.c2[q]);
        }
        {
            // per vector-point: W, b1 in; psi, b2 in when used; out and Wout written; plus the
            // potential rows (and tangent rows) shared by the vectors, and the KB point index.
            const double per = 8.0 * (2 + (a.psi ? 1 : 0) + (a.b2 ? 1 : 0) + 1 + (a.Wout ? 1 : 0));
            double bytes = per * (double)ctx->ng * batch + 4.0 * (double)ctx->ng * vrows * (dvpot ? 2 : 1);
            if (a.kbc) bytes += 4.0 * (double)ctx->ng + 20.0 * (double)ctx->kb.n_sup;
            if (sgw::cluster_plane(n) && ctx->tune[SGW_TUNE_PLANE_VARIANT] == 0) {
                // the row form of the 288 grid: y lines, 36-row step, y lines, each timed on its own
                {
                    Launch Ly(ctx, SGW_PROF_LINES, 1, 16.0 * (double)ctx->ng * batch);
                    sgw::lines288(ctx->W, batch, +1, ctx->tune[SGW_TUNE_LINE_FORM], ctx->tw, st);
                    CKL();
                }
                {
                    Launch L(ctx, SGW_PROF_PLANE_STEP, 1, bytes);
                    sgw::rows36_step(a, batch, ctx->tw, st, ctx->tune[SGW_TUNE_LINE_FORM]);
                    CKL();
                }
                if (a.Wout != nullptr) {
                    Launch Ly(ctx, SGW_PROF_LINES, 1, 16.0 * (double)ctx->ng * batch);
                    sgw::lines288(a.Wout, batch, -1, ctx->tune[SGW_TUNE_LINE_FORM], ctx->tw, st);
                    CKL();
                }
            } else {
                Launch L(ctx, SGW_PROF_PLANE_STEP, 1, bytes);
                sgw::launch_plane_step(n, a, batch, ctx->tw, st, ctx->tune[SGW_TUNE_PLANE_VARIANT],
                                       ctx->tune[SGW_TUNE_LINE_FORM]);
                CKL();
            }
        }
    }
    return SGW_OK;
}

// Per-vector descriptors live in device memory; re-upload only when they change.  The host copy
// kept in the context is the source of the (stream-ordered) copy.
sgw_status upload_info(sgw_ctx* ctx, const std::vector<sgw::VecInfo>& v) {
    if (v.size() <= ctx->info_host.size() &&
        std::memcmp(v.data(), ctx->info_host.data(), sizeof(sgw::VecInfo) * v.size()) == 0)
        return SGW_OK;
    ctx->info_host = v;
    CK(cudaMemcpyAsync(ctx->info, ctx->info_host.data(), sizeof(sgw::VecInfo) * v.size(), cudaMemcpyHostToDevice,
                       ctx->stream));
    return SGW_OK;
}

uint64_t bits(double x) {
    uint64_t u;
    std::memcpy(&u, &x, 8);
    return u;
}

uint64_t fnv(const void* p, size_t n) {
    const unsigned char* c = (const unsigned char*)p;
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    return h;
}

// Run `body` (which only enqueues kernels on the context's stream) directly, or -- in graph
// mode, on a non-default stream, with profiling off -- through a CUDA graph captured on its
// first call with this key and replayed on later calls.
template <class F>
sgw_status graphed(sgw_ctx* ctx, std::vector<uint64_t> key, F&& body) {
    if (!ctx->graph_mode || ctx->prof || ctx->stream == nullptr) return body();
    key.push_back(bits(ctx->emin));
    key.push_back(bits(ctx->emax));
    for (auto& g : ctx->graphs)
        if (g.key == key) {
            CK(cudaGraphLaunch(g.exec, ctx->stream));
            ctx->launches += g.n_launch;
            return SGW_OK;
        }
    const int64_t l0 = ctx->launches;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    sgw_status s = body();
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    if (s != SGW_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    CK(e);
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    if (ctx->graphs.size() >= 8) {
        cudaGraphExecDestroy(ctx->graphs.front().exec);
        ctx->graphs.erase(ctx->graphs.begin());
    }
    ctx->graphs.push_back({key, ex, ctx->launches - l0});
    CK(cudaGraphLaunch(ex, ctx->stream));
    return SGW_OK;
}

void prop_coeffs(sgw_ctx* ctx, double dt, int K, std::vector<cd> c[2], cd phase[2]) {
    const double ebar = 0.5 * (ctx->emax + ctx->emin), de = 0.5 * (ctx->emax - ctx->emin);
    const std::vector<double> J = bessel_j(K, de * std::fabs(dt));
    c[0].resize(K + 1);
    c[1].resize(K + 1);
    cd mi(1.0, 0.0);
    for (int k = 0; k <= K; ++k) {
        const cd v = (k == 0 ? 1.0 : 2.0) * J[k] * mi;      // (2 - delta_k0) (-i)^k J_k
        c[0][k] = dt >= 0 ? v : std::conj(v);
        c[1][k] = std::conj(c[0][k]);
        mi *= cd(0.0, -1.0);
    }
    phase[0] = std::exp(cd(0.0, -ebar * dt));
    phase[1] = std::conj(phase[0]);
}

sgw_status check_ctx(sgw_ctx* ctx, bool need_pot) {
    if (!ctx) return fail(nullptr, SGW_EINVAL, "null context");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return fail(ctx, SGW_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    if (need_pot && !ctx->have_potential) return fail(ctx, SGW_ESTATE, "sgw_set_potential has not been called");
    return SGW_OK;
}

}  // namespace

// =====================================================================================
extern "C" {

const char* sgw_version(void) { return "sgw-gb300 0.1 (sm_103a)"; }

const char* sgw_last_error(const sgw_ctx* ctx) { return ctx ? ctx->err.c_str() : g_setup_err.c_str(); }

sgw_status sgw_setup_grid(sgw_ctx** out, int nx, int ny, int nz, double h, double ecut, int max_batch, int device,
                          void* stream) {
    sgw_ctx* ctx = nullptr;
    if (!out) return fail(nullptr, SGW_EINVAL, "out is null");
    *out = nullptr;
    if (nx != ny || ny != nz || !sgw::grid_supported(nx))
        return fail(nullptr, SGW_EINVAL, "grid must be cubic with n in {16,32,64,128} or {48,96,288}");
    if (!(h > 0) || max_batch < 1) return fail(nullptr, SGW_EINVAL, "h must be > 0 and max_batch >= 1");
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail(nullptr, SGW_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    ctx = new (std::nothrow) sgw_ctx();
    if (!ctx) return fail(nullptr, SGW_ENOMEM, "host allocation failed");
    ctx->n = nx;
    ctx->ng = (int64_t)nx * nx * nx;
    ctx->h = h;
    ctx->dV = h * h * h;
    ctx->L = nx * h;
    ctx->ecut = ecut > 0 ? ecut : 0.0;
    ctx->device = device;
    ctx->stream = (cudaStream_t)stream;
    ctx->max_batch = max_batch;
    const size_t vb = sizeof(float2) * ctx->ng * (size_t)max_batch;
    auto tw = twiddles(nx);
    bool ok = cudaMalloc(&ctx->tw, sizeof(float2) * nx) == cudaSuccess &&
              cudaMalloc(&ctx->vloc, sizeof(float) * ctx->ng) == cudaSuccess &&
              cudaMalloc(&ctx->W, vb) == cudaSuccess && cudaMalloc(&ctx->B1, vb) == cudaSuccess &&
              cudaMalloc(&ctx->B2, vb) == cudaSuccess &&
              cudaMalloc(&ctx->info, sizeof(sgw::VecInfo) * max_batch) == cudaSuccess &&
              cudaMalloc(&ctx->scal, 64 * sizeof(double)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        std::string m = "device allocation failed for " + std::to_string(3.0 * vb / 1e9) + " GB of scratch";
        sgw_destroy(ctx);
        return fail(nullptr, SGW_ENOMEM, m);
    }
    e = cudaMemcpy(ctx->tw, tw.data(), sizeof(float2) * nx, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = sgw::grid_init_attributes(nx);
    if (e == cudaSuccess) e = cudaMemset(ctx->vloc, 0, sizeof(float) * ctx->ng);
    if (e != cudaSuccess) {
        std::string m = std::string("setup: ") + cudaGetErrorString(e);
        sgw_destroy(ctx);
        return fail(nullptr, SGW_ECUDA, m);
    }
    *out = ctx;
    return SGW_OK;
}

void sgw_destroy(sgw_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    free_kb(ctx);
    void* ptrs[] = {ctx->tw, ctx->vloc, ctx->W, ctx->B1, ctx->B2, ctx->info, ctx->scal, ctx->twM};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int i = 0; i < sgw_ctx::kWorkSlots; ++i)
        if (ctx->work[i]) cudaFree(ctx->work[i]);
    for (int k = 0; k < SGW_PROF_KINDS; ++k)
        for (auto& pr : ctx->ev_pending[k]) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    clear_graphs(ctx);
    delete ctx;
}

sgw_status sgw_set_stream(sgw_ctx* ctx, void* stream) {
    if (!ctx) return fail(nullptr, SGW_EINVAL, "null context");
    clear_graphs(ctx);
    ctx->stream = (cudaStream_t)stream;
    return SGW_OK;
}

sgw_status sgw_set_graph_mode(sgw_ctx* ctx, int enable) {
    if (!ctx) return fail(nullptr, SGW_EINVAL, "null context");
    if (!enable) clear_graphs(ctx);
    ctx->graph_mode = enable != 0;
    return SGW_OK;
}

// ---------------------------------------------------------------- split-operator KB factors
// Eigenvalues/vectors of a symmetric n x n matrix (n <= 4) by cyclic Jacobi rotations:
// a = w diag(lam) w^T.
static void jacobi_eig(int n, const double* a_in, double* lam, double* w) {
    double a[16];
    for (int i = 0; i < n * n; ++i) a[i] = a_in[i];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) w[i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                tot += a[i * n + j] * a[i * n + j];
                if (i != j) off += a[i * n + j] * a[i * n + j];
            }
        if (off <= 1e-30 * (tot + 1e-300)) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = a[p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                const double theta = 0.5 * (a[q * n + q] - a[p * n + p]) / apq;
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < n; ++k) {       // columns p, q of a
                    const double akp = a[k * n + p], akq = a[k * n + q];
                    a[k * n + p] = c * akp - sn * akq;
                    a[k * n + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {       // rows p, q
                    const double apk = a[p * n + k], aqk = a[q * n + k];
                    a[p * n + k] = c * apk - sn * aqk;
                    a[q * n + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {       // accumulate the rotation
                    const double wkp = w[k * n + p], wkq = w[k * n + q];
                    w[k * n + p] = c * wkp - sn * wkq;
                    w[k * n + q] = sn * wkp + c * wkq;
                }
            }
    }
    for (int i = 0; i < n; ++i) lam[i] = a[i * n + i];
}

// Q (CGS2, FP64) and M = R E R^T of each atom, the 3D greedy colours of the atoms, uploaded.
static sgw_status build_split_tables(sgw_ctx* ctx, int n_atoms, const int* nproj, const int64_t* sup_off,
                                     const int* sup_idx, const float* beta, const float* e) {
    const int64_t nsup = sup_off[n_atoms];
    const double sdv = std::sqrt(ctx->dV);
    std::vector<float4> q4(std::max<int64_t>(nsup, 1));
    ctx->kb_m.assign((size_t)n_atoms * 16, 0.0);
    for (int a = 0; a < n_atoms; ++a) {
        const int64_t s0 = sup_off[a], ns = sup_off[a + 1] - s0;
        const int P = nproj[a];
        std::vector<double> q((size_t)4 * ns, 0.0);
        double R[16] = {0.0};
        for (int p = 0; p < P; ++p) {
            std::vector<double> v(ns);
            for (int64_t i = 0; i < ns; ++i) v[i] = sdv * beta[4 * (s0 + i) + p];
            for (int pass = 0; pass < 2; ++pass)
                for (int k = 0; k < p; ++k) {
                    double r = 0.0;
                    for (int64_t i = 0; i < ns; ++i) r += q[(size_t)k * ns + i] * v[i];
                    for (int64_t i = 0; i < ns; ++i) v[i] -= r * q[(size_t)k * ns + i];
                    R[k * 4 + p] += r;
                }
            double nrm = 0.0;
            for (int64_t i = 0; i < ns; ++i) nrm += v[i] * v[i];
            nrm = std::sqrt(nrm);
            if (!(nrm > 0.0)) return fail(ctx, SGW_EINVAL, "KB projectors of an atom are linearly dependent");
            R[p * 4 + p] = nrm;
            for (int64_t i = 0; i < ns; ++i) q[(size_t)p * ns + i] = v[i] / nrm;
        }
        for (int64_t i = 0; i < ns; ++i)
            q4[s0 + i] = make_float4((float)q[i], (float)q[(size_t)ns + i], (float)q[(size_t)2 * ns + i],
                                     (float)q[(size_t)3 * ns + i]);
        double* M = &ctx->kb_m[(size_t)a * 16];
        for (int i = 0; i < P; ++i)
            for (int j = 0; j < P; ++j) {
                double m = 0.0;
                for (int k = 0; k < P; ++k) m += R[i * 4 + k] * (double)e[4 * a + k] * R[j * 4 + k];
                M[i * 4 + j] = m;
            }
    }
    // greedy colours: the lowest colour not used by an earlier atom sharing a grid point
    std::vector<uint32_t> mask(ctx->ng, 0u);
    std::vector<int> col(n_atoms, 0);
    int nc = 0;
    for (int a = 0; a < n_atoms; ++a) {
        uint32_t used = 0;
        for (int64_t i = sup_off[a]; i < sup_off[a + 1]; ++i) used |= mask[sup_idx[i]];
        int c = 0;
        while (c < 32 && (used >> c & 1u)) ++c;
        if (c == 32) return fail(ctx, SGW_EINVAL, "more than 32 projector supports overlap at a point");
        for (int64_t i = sup_off[a]; i < sup_off[a + 1]; ++i) mask[sup_idx[i]] |= 1u << c;
        col[a] = c;
        nc = std::max(nc, c + 1);
    }
    std::vector<int> atoms;
    ctx->acol_off.assign(nc + 1, 0);
    for (int c = 0; c < nc; ++c) {
        ctx->acol_off[c] = (int)atoms.size();
        for (int a = 0; a < n_atoms; ++a)
            if (col[a] == c) atoms.push_back(a);
    }
    ctx->acol_off[nc] = (int)atoms.size();
    if (cudaMalloc(&ctx->kbq, sizeof(float4) * q4.size()) != cudaSuccess ||
        cudaMalloc(&ctx->acol_atoms, sizeof(int) * std::max<size_t>(atoms.size(), 1)) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, SGW_ENOMEM, "split-operator table allocation failed");
    }
    CK(cudaMemcpy(ctx->kbq, q4.data(), sizeof(float4) * q4.size(), cudaMemcpyHostToDevice));
    if (!atoms.empty()) CK(cudaMemcpy(ctx->acol_atoms, atoms.data(), sizeof(int) * atoms.size(), cudaMemcpyHostToDevice));
    return SGW_OK;
}

// F_a(tau) = e^{-i tau M_a} - 1 for tau = dt/2 (set 0) and -dt/2 (set 1): the device table of this
// dt (built and uploaded on its first use) in *out
static sgw_status split_factors(sgw_ctx* ctx, double dt, const float2** out) {
    const int na = ctx->kb.n_atoms;
    *out = nullptr;
    if (sgw::rows_path(ctx->n))
        return fail(ctx, SGW_EINVAL, "the split-operator step is built for power-of-two grids only");
    if (na == 0) return SGW_OK;
    for (auto& t : ctx->split_tabs)
        if (t.first == dt) {
            *out = t.second;
            return SGW_OK;
        }
    std::vector<float2> F((size_t)na * 32);
    for (int a = 0; a < na; ++a) {
        double lam[4], w[16];
        jacobi_eig(4, &ctx->kb_m[(size_t)a * 16], lam, w);
        for (int set = 0; set < 2; ++set) {
            const double tau = (set == 0 ? 0.5 : -0.5) * dt;
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) {
                    std::complex<double> f = 0.0;
                    for (int k = 0; k < 4; ++k)
                        f += w[i * 4 + k] * (std::exp(std::complex<double>(0.0, -tau * lam[k])) - 1.0) * w[j * 4 + k];
                    F[((size_t)a * 2 + set) * 16 + i * 4 + j] = make_float2((float)f.real(), (float)f.imag());
                }
        }
    }
    float2* dev = nullptr;
    if (cudaMalloc(&dev, sizeof(float2) * F.size()) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, SGW_ENOMEM, "split-operator factor allocation failed");
    }
    ctx->split_tabs.push_back({dt, dev});
    CK(cudaMemcpyAsync(dev, F.data(), sizeof(float2) * F.size(), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *out = dev;
    return SGW_OK;
}

sgw_status sgw_set_tuning(sgw_ctx* ctx, int key, int value) {
    if (!ctx) return fail(nullptr, SGW_EINVAL, "null context");
    if (key < 0 || key >= SGW_TUNE_KEYS) return fail(ctx, SGW_EINVAL, "unknown tuning key");
    if (value < 0 || (key == SGW_TUNE_PLANE_OPERANDS && value > 3) || (key == SGW_TUNE_PLANE_VARIANT && value > 2) ||
        (key == SGW_TUNE_LINE_FORM && value > 4))
        return fail(ctx, SGW_EINVAL, "tuning value out of range");
    clear_graphs(ctx);
    ctx->tune[key] = value;
    return SGW_OK;
}

sgw_status sgw_get_tuning(sgw_ctx* ctx, int key, int* value_host) {
    if (!ctx) return fail(nullptr, SGW_EINVAL, "null context");
    if (key < 0 || key >= SGW_TUNE_KEYS || !value_host) return fail(ctx, SGW_EINVAL, "bad tuning query");
    *value_host = ctx->tune[key];
    return SGW_OK;
}

sgw_status sgw_autotune(sgw_ctx* ctx, int batch, int reps, int* chosen_host) {
    sgw_status s = check_ctx(ctx, true);
    if (s) return s;
    if (!ctx->have_spectrum) return fail(ctx, SGW_ESTATE, "no spectral interval set");
    if (batch < 1 || batch > ctx->max_batch || reps < 1) return fail(ctx, SGW_EINVAL, "bad autotune arguments");
    void* p = nullptr;
    if ((s = work(ctx, 1, sizeof(float2) * ctx->ng * batch * 2, &p))) return s;
    float2* psi = (float2*)p;
    float2* out = psi + ctx->ng * batch;
    clear_graphs(ctx);
    std::vector<sgw::VecInfo> info(batch, sgw::VecInfo{0, -1, -1, 0});
    if ((s = upload_info(ctx, info))) return s;
    {
        Launch L(ctx, SGW_PROF_OTHER);
        sgw::launch_noise((int)ctx->ng, 0x7u, 0xA7u, 0, 1, batch, (float)(1.0 / std::sqrt(ctx->dV)), psi, ctx->stream);
        CKL();
    }
    std::vector<cd> c[2];
    cd ph[2];
    prop_coeffs(ctx, 0.05, 8, c, ph);
    const std::vector<Step> plan = clenshaw_plan(c, ph, 8);
    int nsm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    const bool prof = ctx->prof;
    ctx->prof = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto timed = [&](float* best_ms) -> sgw_status {
        *best_ms = 1e30f;
        for (int r = 0; r <= reps; ++r) {          // the first run warms up
            cudaEventRecord(e0, ctx->stream);
            sgw_status q = run_series(ctx, plan, psi, out, batch, ctx->vloc, nullptr, ctx->info, false, false);
            if (q) return q;
            cudaEventRecord(e1, ctx->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) return fail(ctx, SGW_ECUDA, "autotune timing failed");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0 && ms < *best_ms) *best_ms = ms;
        }
        return SGW_OK;
    };
    const int order[SGW_TUNE_KEYS] = {SGW_TUNE_PLANE_VARIANT, SGW_TUNE_PLANE_OPERANDS, SGW_TUNE_PLANE_LOOKAHEAD,
                                      SGW_TUNE_PENCIL_LOOKAHEAD, SGW_TUNE_LINE_FORM};
    for (int ki = 0; ki < SGW_TUNE_KEYS && !s; ++ki) {
        const int key = order[ki];
        std::vector<int> cand = {0, 1};
        if (key == SGW_TUNE_PLANE_VARIANT && sgw::plane_pipe_supported(ctx->n)) cand.push_back(2);
        if (key == SGW_TUNE_PLANE_LOOKAHEAD || key == SGW_TUNE_PENCIL_LOOKAHEAD) {
            const int per_sm = key == SGW_TUNE_PLANE_LOOKAHEAD
                                   ? sgw::plane_step_blocks_per_sm(ctx->n, ctx->tune[SGW_TUNE_PLANE_VARIANT], ctx->kb.max_plane_slots)
                                   : sgw::pencil_blocks_per_sm(ctx->n);
            const int R = per_sm * nsm;
            cand = {0, R / 2, R, (3 * R) / 2, 2 * R};
        }
        if (key == SGW_TUNE_LINE_FORM) cand = sgw::cluster_plane(ctx->n) ? std::vector<int>{0, 1, 2, 3, 4}
                                                                          : std::vector<int>{ctx->tune[key]};
        else if (key == SGW_TUNE_PLANE_VARIANT && sgw::cluster_plane(ctx->n)) cand = {0, 1, 2};
        else if (key == SGW_TUNE_PLANE_OPERANDS && sgw::cluster_plane(ctx->n)) cand = {0, 1, 2, 3};
        else if (sgw::rows_path(ctx->n)) cand = {ctx->tune[key]};   // the row kernels take no other launch hints
        int best_v = 0;
        float best = 1e30f;
        for (int v : cand) {
            ctx->tune[key] = v;
            float ms = 0.f;
            if ((s = timed(&ms))) break;
            if (ms < best) {
                best = ms;
                best_v = v;
            }
        }
        ctx->tune[key] = best_v;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->prof = prof;
    if (s) return s;
    if (chosen_host)
        for (int k = 0; k < SGW_TUNE_KEYS; ++k) chosen_host[k] = ctx->tune[k];
    return SGW_OK;
}

sgw_status sgw_set_potential(sgw_ctx* ctx, const float* vloc_dev, int n_atoms, const int* nproj_host,
                             const int64_t* sup_off_host, const int* sup_idx_host, const float* beta_host,
                             const float* e_host) {
    sgw_status s = check_ctx(ctx, false);
    if (s) return s;
    if (!vloc_dev) return fail(ctx, SGW_EINVAL, "vloc_dev is null");
    if (n_atoms < 0) return fail(ctx, SGW_EINVAL, "n_atoms < 0");
    clear_graphs(ctx);
    CK(cudaMemcpyAsync(ctx->vloc, vloc_dev, sizeof(float) * ctx->ng, cudaMemcpyDeviceToDevice, ctx->stream));
    // drop any previous KB data
    CK(cudaStreamSynchronize(ctx->stream));
    free_kb(ctx);
    if (n_atoms > 0) {
        if (!nproj_host || !sup_off_host || !sup_idx_host || !beta_host || !e_host)
            return fail(ctx, SGW_EINVAL, "KB arrays must be non-null when n_atoms > 0");
        if (sup_off_host[0] != 0) return fail(ctx, SGW_EINVAL, "sup_off[0] must be 0");
        for (int a = 0; a < n_atoms; ++a) {
            if (nproj_host[a] < 1 || nproj_host[a] > 4) return fail(ctx, SGW_EINVAL, "nproj must be in 1..4");
            if (sup_off_host[a + 1] < sup_off_host[a]) return fail(ctx, SGW_EINVAL, "sup_off must be non-decreasing");
        }
        const int64_t nsup = sup_off_host[n_atoms];
        if (nsup > INT32_MAX) return fail(ctx, SGW_EINVAL, "too many support points");
        for (int64_t i = 0; i < nsup; ++i)
            if (sup_idx_host[i] < 0 || sup_idx_host[i] >= ctx->ng) return fail(ctx, SGW_EINVAL, "support index out of range");
        for (int a = 0; a < n_atoms; ++a)
            for (int64_t i = sup_off_host[a] + 1; i < sup_off_host[a + 1]; ++i)
                if (sup_idx_host[i] <= sup_idx_host[i - 1])
                    return fail(ctx, SGW_EINVAL, "each atom's support indices must be strictly increasing");
        std::vector<float4> sup_beta(std::max<int64_t>(nsup, 1)), atom_e(n_atoms);
        for (int a = 0; a < n_atoms; ++a) {
            atom_e[a] = make_float4(e_host[4 * a], e_host[4 * a + 1], e_host[4 * a + 2], e_host[4 * a + 3]);
            for (int64_t i = sup_off_host[a]; i < sup_off_host[a + 1]; ++i) {
                float4 b = make_float4(beta_host[4 * i], beta_host[4 * i + 1], beta_host[4 * i + 2], beta_host[4 * i + 3]);
                if (nproj_host[a] < 4) b.w = 0.f;
                if (nproj_host[a] < 3) b.z = 0.f;
                if (nproj_host[a] < 2) b.y = 0.f;
                sup_beta[i] = b;
            }
        }
        // slots: one per (unit, atom) pair where the atom's support meets the unit (a unit is an xy
        // plane on the plane path, 8 x rows on the row path: unit_points consecutive points); atom a's
        // points in unit z are one contiguous run of its sorted support: [run_beg, run_end)
        const int n = ctx->n;
        const int64_t plane_sz = sgw::unit_points(n);
        const int nu = (int)(ctx->ng / plane_sz);
        if (plane_sz > 65536) return fail(ctx, SGW_EINVAL, "in-unit offsets must fit 16 bits");
        std::vector<std::vector<int>> plane_atoms(nu);
        std::vector<std::vector<std::pair<int64_t, int64_t>>> plane_runs(nu);
        for (int a = 0; a < n_atoms; ++a) {
            int64_t i = sup_off_host[a];
            while (i < sup_off_host[a + 1]) {
                const int z = (int)(sup_idx_host[i] / plane_sz);
                int64_t j = i;
                while (j < sup_off_host[a + 1] && sup_idx_host[j] / plane_sz == z) ++j;
                plane_atoms[z].push_back(a);
                plane_runs[z].push_back({i, j});
                i = j;
            }
        }
        std::vector<int> plane_off(nu + 1, 0);
        int max_slots = 0;
        for (int z = 0; z < nu; ++z) {
            plane_off[z + 1] = plane_off[z] + (int)plane_atoms[z].size();
            max_slots = std::max(max_slots, (int)plane_atoms[z].size());
        }
        const int total_slots = plane_off[nu];
        if (max_slots >= 65536) return fail(ctx, SGW_EINVAL, "too many projector supports meet one plane");
        const size_t smem = sgw::plane_step_smem(n, max_slots);
        int optin = 0;
        CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
        if (smem > (size_t)optin || (sgw::plane_pipe_supported(n) && sgw::plane_pipe_smem(n, max_slots) > (size_t)optin))
            return fail(ctx, SGW_EINVAL, "the projector slots of one plane do not fit in shared memory");
        CK(sgw::plane_step_reserve_smem(n, max_slots));
        std::vector<int> slot_atom(std::max(total_slots, 1));
        std::vector<std::vector<int>> atom_slots(n_atoms);
        for (int z = 0; z < nu; ++z)
            for (int k = 0; k < (int)plane_atoms[z].size(); ++k) {
                slot_atom[plane_off[z] + k] = plane_atoms[z][k];
                atom_slots[plane_atoms[z][k]].push_back(plane_off[z] + k);
            }
        std::vector<int> atom_pos_off(n_atoms + 1, 0), atom_pos;
        for (int a = 0; a < n_atoms; ++a) {
            atom_pos_off[a + 1] = atom_pos_off[a] + (int)atom_slots[a].size();
            atom_pos.insert(atom_pos.end(), atom_slots[a].begin(), atom_slots[a].end());
        }
        // colour the slots of each unit greedily (lowest colour not used by an overlapping slot)
        std::vector<int> slot_col(std::max(total_slots, 1), 0);
        int max_colors = 0;
        std::vector<uint32_t> mask(plane_sz);
        for (int z = 0; z < nu; ++z) {
            std::fill(mask.begin(), mask.end(), 0u);
            for (int k = 0; k < (int)plane_atoms[z].size(); ++k) {
                uint32_t used = 0;
                for (int64_t i = plane_runs[z][k].first; i < plane_runs[z][k].second; ++i)
                    used |= mask[sup_idx_host[i] - z * plane_sz];
                int c = 0;
                while (c < 32 && (used >> c & 1u)) ++c;
                if (c == 32) return fail(ctx, SGW_EINVAL, "more than 32 projector supports overlap at a point");
                for (int64_t i = plane_runs[z][k].first; i < plane_runs[z][k].second; ++i)
                    mask[sup_idx_host[i] - z * plane_sz] |= 1u << c;
                slot_col[plane_off[z] + k] = c;
                max_colors = std::max(max_colors, c + 1);
            }
        }
        // unit-major, colour-major, slot-major entry table
        std::vector<int> kbe_col((size_t)nu * (max_colors + 1), 0);
        std::vector<unsigned> kbe_os;
        std::vector<float4> kbe_beta;
        kbe_os.reserve(nsup);
        kbe_beta.reserve(nsup);
        std::vector<int> kbe_slot_beg(std::max(total_slots, 1)), kbe_slot_end(std::max(total_slots, 1));
        for (int z = 0; z < nu; ++z) {
            for (int c = 0; c < max_colors; ++c) {
                kbe_col[(size_t)z * (max_colors + 1) + c] = (int)kbe_os.size();
                for (int k = 0; k < (int)plane_atoms[z].size(); ++k) {
                    if (slot_col[plane_off[z] + k] != c) continue;
                    kbe_slot_beg[plane_off[z] + k] = (int)kbe_os.size();
                    for (int64_t i = plane_runs[z][k].first; i < plane_runs[z][k].second; ++i) {
                        kbe_os.push_back((unsigned)(sup_idx_host[i] - z * plane_sz) | ((unsigned)k << 16));
                        kbe_beta.push_back(sup_beta[i]);
                    }
                    kbe_slot_end[plane_off[z] + k] = (int)kbe_os.size();
                }
            }
            kbe_col[(size_t)z * (max_colors + 1) + max_colors] = (int)kbe_os.size();
        }
        sgw::KBDev& kb = ctx->kb;
        kb.total_slots = total_slots;
        kb.max_plane_slots = max_slots;
        kb.max_colors = max_colors;
        kb.n_atoms = n_atoms;
        kb.n_proj = 4 * n_atoms;
        kb.n_sup = nsup;
        const size_t ns1 = std::max<int64_t>(nsup, 1), ts1 = std::max(total_slots, 1);
        bool ok = cudaMalloc(&kb.atom_nproj, sizeof(int) * n_atoms) == cudaSuccess &&
                  cudaMalloc(&kb.atom_off, sizeof(int64_t) * (n_atoms + 1)) == cudaSuccess &&
                  cudaMalloc(&kb.sup_idx, sizeof(int) * ns1) == cudaSuccess &&
                  cudaMalloc(&kb.sup_beta, sizeof(float4) * ns1) == cudaSuccess &&
                  cudaMalloc(&kb.atom_e, sizeof(float4) * n_atoms) == cudaSuccess &&
                  cudaMalloc(&kb.plane_off, sizeof(int) * (nu + 1)) == cudaSuccess &&
                  cudaMalloc(&kb.slot_atom, sizeof(int) * ts1) == cudaSuccess &&
                  cudaMalloc(&kb.kbe_col, sizeof(int) * kbe_col.size()) == cudaSuccess &&
                  cudaMalloc(&kb.kbe_os, sizeof(unsigned) * ns1) == cudaSuccess &&
                  cudaMalloc(&kb.kbe_beta, sizeof(float4) * ns1) == cudaSuccess &&
                  cudaMalloc(&kb.kbe_slot_beg, sizeof(int) * ts1) == cudaSuccess &&
                  cudaMalloc(&kb.kbe_slot_end, sizeof(int) * ts1) == cudaSuccess &&
                  cudaMalloc(&kb.atom_pos_off, sizeof(int) * (n_atoms + 1)) == cudaSuccess &&
                  cudaMalloc(&kb.atom_pos, sizeof(int) * ts1) == cudaSuccess &&
                  cudaMalloc(&ctx->kbc, sizeof(float2) * (size_t)kb.n_proj * ctx->max_batch) == cudaSuccess &&
                  cudaMalloc(&ctx->kbp, sizeof(float2) * 4 * ts1 * ctx->max_batch) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            free_kb(ctx);
            return fail(ctx, SGW_ENOMEM, "KB device allocation failed");
        }
        CK(cudaMemcpy(kb.atom_nproj, nproj_host, sizeof(int) * n_atoms, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(kb.atom_off, sup_off_host, sizeof(int64_t) * (n_atoms + 1), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(kb.sup_idx, sup_idx_host, sizeof(int) * nsup, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(kb.sup_beta, sup_beta.data(), sizeof(float4) * nsup, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(kb.atom_e, atom_e.data(), sizeof(float4) * n_atoms, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(kb.plane_off, plane_off.data(), sizeof(int) * (nu + 1), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(kb.slot_atom, slot_atom.data(), sizeof(int) * ts1, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(kb.kbe_col, kbe_col.data(), sizeof(int) * kbe_col.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(kb.kbe_os, kbe_os.data(), sizeof(unsigned) * nsup, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(kb.kbe_beta, kbe_beta.data(), sizeof(float4) * nsup, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(kb.kbe_slot_beg, kbe_slot_beg.data(), sizeof(int) * ts1, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(kb.kbe_slot_end, kbe_slot_end.data(), sizeof(int) * ts1, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(kb.atom_pos_off, atom_pos_off.data(), sizeof(int) * (n_atoms + 1), cudaMemcpyHostToDevice));
        if (total_slots > 0)
            CK(cudaMemcpy(kb.atom_pos, atom_pos.data(), sizeof(int) * total_slots, cudaMemcpyHostToDevice));
        if ((s = build_split_tables(ctx, n_atoms, nproj_host, sup_off_host, sup_idx_host, beta_host, e_host)))
            return s;
    }
    ctx->have_potential = true;
    return SGW_OK;
}

sgw_status sgw_apply_h(sgw_ctx* ctx, const void* in_dev, void* out_dev, int batch) {
    sgw_status s = check_ctx(ctx, true);
    if (s) return s;
    if (batch < 0 || batch > ctx->max_batch) return fail(ctx, SGW_EINVAL, "batch out of range");
    if (batch == 0) return SGW_OK;
    if (!in_dev || !out_dev || in_dev == out_dev) return fail(ctx, SGW_EINVAL, "bad in/out pointers");
    SGW_ALIGNED(ctx, in_dev, out_dev);
    std::vector<sgw::VecInfo> info(batch, sgw::VecInfo{0, -1, -1, 0});
    if ((s = upload_info(ctx, info))) return s;
    const float kscale = (float)std::pow(2.0 * M_PI / ctx->L, 2);
    const float2* in = (const float2*)in_dev;
    {
        Launch L(ctx, SGW_PROF_PLANE_FWD);
        sgw::launch_plane_fwd(ctx->n, in, ctx->W, batch, ctx->tw, ctx->stream);
        CKL();
    }
    if (ctx->kb.n_atoms > 0) {
        Launch L(ctx, SGW_PROF_KB);
        sgw::launch_kb_project(ctx->n, ctx->kb, in, batch, (float)ctx->dV, ctx->kbc, ctx->stream);
        CKL();
    }
    {
        Launch L(ctx, SGW_PROF_PENCIL);
        sgw::launch_pencil(ctx->n, ctx->W, batch, 0, kscale, (float)ctx->ecut, ctx->tw, ctx->stream,
                           ctx->tune[SGW_TUNE_PENCIL_LOOKAHEAD], nullptr, 0.f, ctx->tune[SGW_TUNE_LINE_FORM]);
        CKL();
    }
    sgw::StepArgs a{};
    a.W = ctx->W;
    a.Wout = nullptr;
    a.b1 = in;
    a.out = (float2*)out_dev;
    a.vpot = ctx->vloc;
    a.info = ctx->info;
    a.kbc = ctx->kb.n_atoms > 0 ? ctx->kbc : nullptr;
    set_kb_args(ctx, a);
    a.kbp = nullptr;
    a.n_proj = ctx->kb.n_proj;
    a.ebar = 0.f;
    a.alpha = 1.f;
    a.pf_ahead = ctx->tune[SGW_TUNE_PLANE_LOOKAHEAD];
    a.pf_operands = ctx->tune[SGW_TUNE_PLANE_OPERANDS];
    for (int q = 0; q < 2; ++q) {
        a.coef.cpsi[q] = make_float2(0.f, 0.f);
        a.coef.ch[q] = make_float2(1.f, 0.f);
        a.coef.c2[q] = make_float2(0.f, 0.f);
    }
    {
        Launch L(ctx, SGW_PROF_PLANE_STEP);
        sgw::launch_plane_step(ctx->n, a, batch, ctx->tw, ctx->stream, ctx->tune[SGW_TUNE_PLANE_VARIANT],
                               ctx->tune[SGW_TUNE_LINE_FORM]);
        CKL();
    }
    return SGW_OK;
}

sgw_status sgw_set_spectrum(sgw_ctx* ctx, double emin, double emax) {
    if (!ctx) return fail(nullptr, SGW_EINVAL, "null context");
    if (!(emax > emin)) return fail(ctx, SGW_EINVAL, "emax must exceed emin");
    ctx->emin = emin;
    ctx->emax = emax;
    ctx->have_spectrum = true;
    return SGW_OK;
}

sgw_status sgw_spectral_bounds(sgw_ctx* ctx, int n_iter, uint64_t seed, double margin, double* emin_host,
                               double* emax_host, double* raw_host) {
    sgw_status s = check_ctx(ctx, true);
    if (s) return s;
    if (n_iter < 1 || !emin_host || !emax_host || !(margin >= 0))
        return fail(ctx, SGW_EINVAL, "bad spectral-bounds arguments");
    cudaStream_t st = ctx->stream;
    float2 *v, *w;
    void* p;
    if ((s = work(ctx, 0, sizeof(float2) * ctx->ng * 2, &p))) return s;
    v = (float2*)p;
    w = v + ctx->ng;
    double* est = ctx->scal + 8;   // est[0] E_max estimate, est[1] shifted estimate
    sgw::launch_noise((int)ctx->ng, seed, 0xB0B0u, 0, 1, 1, (float)(1.0 / std::sqrt(ctx->dV)), v, st);
    CKL();
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            sgw::launch_noise((int)ctx->ng, seed, 0xB0B0u, 0, 1, 1, (float)(1.0 / std::sqrt(ctx->dV)), v, st);
            CKL();
        }
        for (int it = 0; it < n_iter; ++it) {
            if ((s = sgw_apply_h(ctx, v, w, 1))) return s;
            Launch L(ctx, SGW_PROF_OTHER, 2);
            sgw::launch_dot2((int)ctx->ng, v, w, ctx->scal, st);
            CKL();
            sgw::launch_power_update((int)ctx->ng, w, v, ctx->scal, est + pass, pass == 1 ? est : nullptr,
                                     (float)ctx->dV, st);
            CKL();
        }
    }
    double e[2];
    CK(cudaMemcpyAsync(e, est, sizeof(e), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const double emax = e[0], emin = e[0] + e[1];
    if (raw_host) {
        raw_host[0] = emin;
        raw_host[1] = emax;
    }
    const double wd = emax - emin;
    *emin_host = emin - margin * wd;
    *emax_host = emax + margin * wd;
    return sgw_set_spectrum(ctx, *emin_host, *emax_host);
}

sgw_status sgw_gapped_filter_coeffs(double e_homo, double e_lumo, double emin, double emax, int n_cheb, double ridge,
                                    double* coeffs_host) {
    sgw_ctx* ctx = nullptr;
    if (!coeffs_host || n_cheb < 0 || !(emax > emin) || !(e_lumo >= e_homo) || !(ridge > 0))
        return fail(ctx, SGW_EINVAL, "bad gapped-filter arguments");
    const double ebar = 0.5 * (emax + emin), de = 0.5 * (emax - emin);
    const double xh = (e_homo - ebar) / de, xl = (e_lumo - ebar) / de;
    const int N1 = n_cheb + 1;
    const int M = 4 * N1;
    // Over all M Chebyshev-Gauss nodes sum_m T_j T_k = D_jj delta_jk (D_00 = M, D_jj = M/2): the normal
    // matrix of the fit without the gap nodes is D + rho - U^T U, U the rows of the gap nodes.  Solve it
    // through the Woodbury identity with the small capacitance matrix I - U D'^-1 U^T (Cholesky).
    std::vector<double> dinv(N1), rhs(N1, 0.0), Tk(N1);
    const double rho = ridge * M;
    for (int k = 0; k < N1; ++k) dinv[k] = 1.0 / ((k == 0 ? (double)M : 0.5 * M) + rho);
    std::vector<std::vector<double>> U;
    for (int m = 0; m < M; ++m) {
        const double th = M_PI * (m + 0.5) / M;
        const double x = std::cos(th);
        const bool keep = (x <= xh) || (x >= xl);
        for (int k = 0; k < N1; ++k) Tk[k] = std::cos(k * th);
        if (keep) {
            if (x <= xh)
                for (int k = 0; k < N1; ++k) rhs[k] += Tk[k];
        } else {
            U.push_back(Tk);
        }
    }
    const int G = (int)U.size();
    // y = D'^-1 rhs
    std::vector<double> y(N1);
    for (int k = 0; k < N1; ++k) y[k] = dinv[k] * rhs[k];
    if (G > 0) {
        // C = I - U D'^-1 U^T ; solve C z = U y ; a = y + D'^-1 U^T z
        std::vector<double> C((size_t)G * G), z(G);
        for (int i = 0; i < G; ++i) {
            for (int j = 0; j <= i; ++j) {
                double acc = 0;
                for (int k = 0; k < N1; ++k) acc += U[i][k] * dinv[k] * U[j][k];
                C[(size_t)i * G + j] = C[(size_t)j * G + i] = (i == j ? 1.0 : 0.0) - acc;
            }
            double acc = 0;
            for (int k = 0; k < N1; ++k) acc += U[i][k] * y[k];
            z[i] = acc;
        }
        // Cholesky C = L L^T (C is positive definite because the regularised normal matrix is)
        for (int j = 0; j < G; ++j) {
            double d = C[(size_t)j * G + j];
            for (int k = 0; k < j; ++k) d -= C[(size_t)j * G + k] * C[(size_t)j * G + k];
            if (!(d > 0)) return fail(ctx, SGW_ENOCONV, "gapped-filter capacitance matrix is not positive definite");
            d = std::sqrt(d);
            C[(size_t)j * G + j] = d;
            for (int i = j + 1; i < G; ++i) {
                double t = C[(size_t)i * G + j];
                for (int k = 0; k < j; ++k) t -= C[(size_t)i * G + k] * C[(size_t)j * G + k];
                C[(size_t)i * G + j] = t / d;
            }
        }
        for (int i = 0; i < G; ++i) {  // forward
            double t = z[i];
            for (int k = 0; k < i; ++k) t -= C[(size_t)i * G + k] * z[k];
            z[i] = t / C[(size_t)i * G + i];
        }
        for (int i = G - 1; i >= 0; --i) {  // backward
            double t = z[i];
            for (int k = i + 1; k < G; ++k) t -= C[(size_t)k * G + i] * z[k];
            z[i] = t / C[(size_t)i * G + i];
        }
        for (int k = 0; k < N1; ++k) {
            double acc = 0;
            for (int i = 0; i < G; ++i) acc += U[i][k] * z[i];
            y[k] += dinv[k] * acc;
        }
    }
    for (int k = 0; k < N1; ++k) coeffs_host[k] = y[k];
    return SGW_OK;
}

sgw_status sgw_propagator_coeffs(double emin, double emax, double dt, int cheb_deg, double* coeffs_host,
                                 double* phase_host) {
    if (!coeffs_host || !phase_host || cheb_deg < 0 || !(emax > emin))
        return fail(nullptr, SGW_EINVAL, "bad propagator-coefficient arguments");
    sgw_ctx tmp;
    tmp.emin = emin;
    tmp.emax = emax;
    std::vector<cd> c[2];
    cd ph[2];
    prop_coeffs(&tmp, dt, cheb_deg, c, ph);
    for (int k = 0; k <= cheb_deg; ++k) {
        coeffs_host[2 * k] = c[0][k].real();
        coeffs_host[2 * k + 1] = c[0][k].imag();
    }
    phase_host[0] = ph[0].real();
    phase_host[1] = ph[0].imag();
    return SGW_OK;
}

sgw_status sgw_filter_occupied(sgw_ctx* ctx, const double* coeffs_host, int n_cheb, const void* in_dev, void* out_dev,
                               int batch) {
    sgw_status s = check_ctx(ctx, true);
    if (s) return s;
    if (!ctx->have_spectrum) return fail(ctx, SGW_ESTATE, "no spectral interval set");
    if (!coeffs_host || n_cheb < 0 || batch < 0 || batch > ctx->max_batch || (batch > 0 && (!in_dev || !out_dev)))
        return fail(ctx, SGW_EINVAL, "bad filter arguments");
    if (batch == 0) return SGW_OK;
    SGW_ALIGNED(ctx, in_dev, out_dev);
    std::vector<cd> c[2];
    c[0].assign(coeffs_host, coeffs_host + n_cheb + 1);
    c[1] = c[0];
    const cd one[2] = {1.0, 1.0};
    if (n_cheb == 0) {
        // out = a_0 in : run an empty plan then scale on the host side would need a kernel; use K=1 with c1=0
        c[0].push_back(0.0);
        c[1].push_back(0.0);
        n_cheb = 1;
    }
    const std::vector<Step> plan = clenshaw_plan(c, one, n_cheb);
    std::vector<sgw::VecInfo> info(batch, sgw::VecInfo{0, -1, -1, 0});
    if ((s = upload_info(ctx, info))) return s;
    std::vector<uint64_t> key = {1, (uint64_t)n_cheb, (uint64_t)batch, (uint64_t)in_dev, (uint64_t)out_dev,
                                 fnv(coeffs_host, sizeof(double) * (n_cheb + 1))};
    return graphed(ctx, key, [&]() {
        return run_series(ctx, plan, (const float2*)in_dev, (float2*)out_dev, batch, ctx->vloc, nullptr, ctx->info,
                          false, false);
    });
}

sgw_status sgw_white_noise(sgw_ctx* ctx, uint64_t seed, uint32_t stream_id, int sample0, int n_samples, int n_vec,
                           void* out_dev) {
    sgw_status s = check_ctx(ctx, false);
    if (s) return s;
    if (n_samples < 0 || n_vec < 0 || sample0 < 0 || (!out_dev && n_samples * n_vec > 0))
        return fail(ctx, SGW_EINVAL, "bad noise arguments");
    Launch L(ctx, SGW_PROF_OTHER);
    sgw::launch_noise((int)ctx->ng, seed, stream_id, sample0, n_samples, n_vec, (float)(1.0 / std::sqrt(ctx->dV)),
                      (float2*)out_dev, ctx->stream);
    CKL();
    return SGW_OK;
}

sgw_status sgw_prepare_sample(sgw_ctx* ctx, const void* noise_dev, const void* filt_dev, const float* phi_dev,
                              int n_samples, int n_eta, void* eta_dev, void* zeta_dev, float* source_dev) {
    sgw_status s = check_ctx(ctx, false);
    if (s) return s;
    if (n_samples < 0 || n_eta < 1) return fail(ctx, SGW_EINVAL, "bad prepare arguments");
    if (n_samples == 0) return SGW_OK;
    if (!noise_dev || !filt_dev || !phi_dev || !eta_dev || !zeta_dev || !source_dev)
        return fail(ctx, SGW_EINVAL, "null prepare pointers");
    SGW_ALIGNED(ctx, noise_dev, filt_dev, phi_dev, eta_dev, zeta_dev, source_dev);
    Launch L(ctx, SGW_PROF_OTHER);
    sgw::launch_prepare((int)ctx->ng, (const float2*)noise_dev, (const float2*)filt_dev, phi_dev, n_samples, n_eta,
                        (float2*)eta_dev, (float2*)zeta_dev, source_dev, ctx->stream);
    CKL();
    return SGW_OK;
}

sgw_status sgw_propagate(sgw_ctx* ctx, void* psi_dev, int batch, int n_steps, double dt, int cheb_deg,
                         const int8_t* dir_host) {
    sgw_status s = check_ctx(ctx, true);
    if (s) return s;
    if (!ctx->have_spectrum) return fail(ctx, SGW_ESTATE, "no spectral interval set");
    if (batch < 0 || batch > ctx->max_batch || n_steps < 0 || cheb_deg < 1 || (!psi_dev && batch > 0))
        return fail(ctx, SGW_EINVAL, "bad propagate arguments");
    if (batch == 0 || n_steps == 0) return SGW_OK;
    SGW_ALIGNED(ctx, psi_dev);
    std::vector<cd> c[2];
    cd ph[2];
    prop_coeffs(ctx, dt, cheb_deg, c, ph);
    const std::vector<Step> plan = clenshaw_plan(c, ph, cheb_deg);
    std::vector<sgw::VecInfo> info(batch, sgw::VecInfo{0, -1, -1, 0});
    if (dir_host)
        for (int b = 0; b < batch; ++b) {
            if (dir_host[b] != 1 && dir_host[b] != -1) return fail(ctx, SGW_EINVAL, "dir must be +1 or -1");
            info[b].cset = dir_host[b] > 0 ? 0 : 1;
        }
    if ((s = upload_info(ctx, info))) return s;
    float2* psi = (float2*)psi_dev;
    std::vector<uint64_t> key = {2, (uint64_t)batch, (uint64_t)n_steps, bits(dt), (uint64_t)cheb_deg, (uint64_t)psi,
                                 fnv(info.data(), sizeof(sgw::VecInfo) * info.size())};
    return graphed(ctx, key, [&]() {
        for (int j = 0; j < n_steps; ++j) {
            sgw_status r = run_series(ctx, plan, psi, psi, batch, ctx->vloc, nullptr, ctx->info, j > 0, j + 1 < n_steps);
            if (r) return r;
        }
        return SGW_OK;
    });
}

// One split-operator step of a batch in place (ctx->info: per-vector direction, potential row,
// tangent row and partner); split_factors(ctx, dt) must have run.
static sgw_status split_step_batch(sgw_ctx* ctx, float2* psi, int batch, const float* vpot, const float* dvpot,
                                   double dt, const float2* F) {
    const int n = ctx->n;
    const float kscale = (float)std::pow(2.0 * M_PI / ctx->L, 2);
    const int nc = (int)ctx->acol_off.size() - 1;
    const double vb = (double)ctx->ng * batch;
    const double kb_bytes = (double)ctx->kb.n_sup * batch * 24.0;     // gather + write back + Q per point
    auto kb_half = [&](bool descending) -> sgw_status {
        for (int i = 0; i < nc; ++i) {
            const int c = descending ? nc - 1 - i : i;
            const int a0 = ctx->acol_off[c], na = ctx->acol_off[c + 1] - a0;
            Launch L(ctx, SGW_PROF_KB, 1, kb_bytes * na / std::max(ctx->kb.n_atoms, 1));
            sgw::launch_kb_split(ctx->acol_atoms + a0, na, ctx->kb, ctx->kbq, F, ctx->info, psi, batch,
                                 (size_t)ctx->ng, ctx->stream);
            CKL();
        }
        return SGW_OK;
    };
    sgw_status r;
    if (ctx->kb.n_atoms > 0 && (r = kb_half(false))) return r;
    {
        Launch L(ctx, SGW_PROF_PLANE_FWD, 1, (dvpot ? 24.0 : 16.0) * vb + 8.0 * ctx->ng);
        sgw::launch_plane_fwd_phase(n, psi, vpot, dvpot, ctx->info, (float)dt, ctx->W, batch, ctx->tw, ctx->stream);
        CKL();
    }
    {
        Launch L(ctx, SGW_PROF_PENCIL, 1, 16.0 * vb);
        sgw::launch_pencil(n, ctx->W, batch, 2, kscale, (float)ctx->ecut, ctx->tw, ctx->stream,
                           ctx->tune[SGW_TUNE_PENCIL_LOOKAHEAD], ctx->info, (float)dt);
        CKL();
    }
    {
        Launch L(ctx, SGW_PROF_SPLIT_INV, 1, 16.0 * vb + 4.0 * ctx->ng);
        sgw::launch_plane_inv_phase(n, ctx->W, vpot, ctx->info, (float)dt, psi, batch, ctx->tw, ctx->stream);
        CKL();
    }
    if (dvpot != nullptr) {
        Launch L(ctx, SGW_PROF_OTHER, 1, 14.0 * vb);     // tangent halves: own + partner + dv
        sgw::launch_split_tangent(psi, dvpot, ctx->info, (float)dt, batch, ctx->ng, ctx->stream);
        CKL();
    }
    if (ctx->kb.n_atoms > 0 && (r = kb_half(true))) return r;
    return SGW_OK;
}

sgw_status sgw_propagate_split(sgw_ctx* ctx, void* psi_dev, int batch, int n_steps, double dt,
                               const int8_t* dir_host) {
    sgw_status s = check_ctx(ctx, true);
    if (s) return s;
    if (batch < 0 || batch > ctx->max_batch || n_steps < 0 || (!psi_dev && batch > 0))
        return fail(ctx, SGW_EINVAL, "bad split-propagate arguments");
    if (batch == 0 || n_steps == 0) return SGW_OK;
    SGW_ALIGNED(ctx, psi_dev);
    std::vector<sgw::VecInfo> info(batch, sgw::VecInfo{0, -1, -1, 0});
    if (dir_host)
        for (int b = 0; b < batch; ++b) {
            if (dir_host[b] != 1 && dir_host[b] != -1) return fail(ctx, SGW_EINVAL, "dir must be +1 or -1");
            info[b].cset = dir_host[b] > 0 ? 0 : 1;
        }
    if ((s = upload_info(ctx, info))) return s;
    const float2* F = nullptr;
    if ((s = split_factors(ctx, dt, &F))) return s;
    float2* psi = (float2*)psi_dev;
    std::vector<uint64_t> key = {7, (uint64_t)batch, (uint64_t)n_steps, bits(dt), (uint64_t)psi,
                                 fnv(info.data(), sizeof(sgw::VecInfo) * info.size())};
    return graphed(ctx, key, [&]() {
        for (int j = 0; j < n_steps; ++j)
            if (sgw_status r = split_step_batch(ctx, psi, batch, ctx->vloc, nullptr, dt, F)) return r;
        return SGW_OK;
    });
}

// The xi basis of a call: per-sample Philox draws (seed, stream, sample0 + s), K segment draws of L
// points per function, scale c = 1 / sqrt(n_xi K L dV / N_g).
struct XiArgs {
    uint64_t seed;
    uint32_t stream;
    int sample0, n_xi, K, L;
    double c;
};

static sgw_status xi_args(sgw_ctx* ctx, uint64_t seed, uint32_t stream, int sample0, int n_xi, double f_g, int L,
                          XiArgs* xa) {
    if (n_xi < 1 || !(f_g > 0.0) || L < 1 || L > 32 || ctx->ng % L != 0 || sample0 < 0)
        return fail(ctx, SGW_EINVAL, "bad xi arguments (n_xi >= 1, f_g > 0, 1 <= L <= 32 dividing N_g)");
    xa->seed = seed;
    xa->stream = stream;
    xa->sample0 = sample0;
    xa->n_xi = n_xi;
    xa->L = L;
    xa->K = (int)std::max<long long>(1, std::llround((double)ctx->ng * f_g / L));
    xa->c = 1.0 / std::sqrt((double)n_xi * xa->K * L * ctx->dV / (double)ctx->ng);
    return SGW_OK;
}

static sgw_status tdh_run(sgw_ctx* ctx, const void* eta_dev, const float* source_dev, int n_samples, int n_eta,
                          int n_steps, double dt, int cheb_deg, double weight, float* uR_dev, const XiArgs* xi) {
    sgw_status s = check_ctx(ctx, true);
    if (s) return s;
    if (cheb_deg > 0 && !ctx->have_spectrum) return fail(ctx, SGW_ESTATE, "no spectral interval set");
    if (n_samples < 0 || n_eta < 1 || n_steps < 0 || cheb_deg < 0 || 2LL * n_samples * n_eta > ctx->max_batch)
        return fail(ctx, SGW_EINVAL, "bad TDH arguments (2 n_samples n_eta must be <= max_batch)");
    if (n_samples == 0) return SGW_OK;
    if (!eta_dev || !source_dev || !uR_dev) return fail(ctx, SGW_EINVAL, "null TDH pointers");
    SGW_ALIGNED(ctx, eta_dev, source_dev, uR_dev);
    cudaStream_t st = ctx->stream;
    const int n = ctx->n;
    const int64_t ng = ctx->ng;
    const int B = 2 * n_samples * n_eta;
    const float w = (float)(weight > 0 ? weight : 2.0 / n_eta);
    const float kscale = (float)std::pow(2.0 * M_PI / ctx->L, 2);
    void *p0, *p1, *p2;
    if ((s = work(ctx, 1, sizeof(float2) * ng * B, &p0))) return s;                 // psi batch
    if ((s = work(ctx, 2, sizeof(float2) * ng * n_samples, &p1))) return s;         // Poisson planes
    if ((s = work(ctx, 3, sizeof(float) * ng * n_samples * 4, &p2))) return s;      // vtot, dv, rho0, vp
    float2* psi = (float2*)p0;
    float2* Wp = (float2*)p1;
    float* vtot = (float*)p2;
    float* dv = vtot + ng * n_samples;
    float* rho0 = dv + ng * n_samples;
    float* vp = rho0 + ng * n_samples;
    std::vector<sgw::VecInfo> info(B);
    for (int sm = 0; sm < n_samples; ++sm)
        for (int l = 0; l < 2 * n_eta; ++l) {
            const int b = sm * 2 * n_eta + l;
            const bool tan = l >= n_eta;
            info[b] = sgw::VecInfo{sm, tan ? sm : -1, tan ? b - n_eta : -1, 0};
        }
    if ((s = upload_info(ctx, info))) return s;
    std::vector<cd> c[2];
    cd ph[2];
    std::vector<Step> plan;
    const float2* F = nullptr;
    if (cheb_deg > 0) {
        prop_coeffs(ctx, dt, cheb_deg, c, ph);
        plan = clenshaw_plan(c, ph, cheb_deg);
    } else if ((s = split_factors(ctx, dt, &F))) {
        return s;
    }
    const int64_t uR_stride = (int64_t)(n_steps + 1) * ng;
    std::vector<uint64_t> key = {3, (uint64_t)n_samples, (uint64_t)n_eta, (uint64_t)n_steps, bits(dt),
                                 (uint64_t)cheb_deg, bits(w), (uint64_t)eta_dev, (uint64_t)source_dev, (uint64_t)uR_dev,
                                 (uint64_t)psi, (uint64_t)Wp, (uint64_t)vtot};
    if (xi) {
        key.insert(key.end(), {xi->seed, (uint64_t)xi->stream, (uint64_t)xi->sample0, (uint64_t)xi->n_xi,
                               (uint64_t)xi->K, (uint64_t)xi->L});
    }
    return graphed(ctx, key, [&]() -> sgw_status {
        // v_p = v_C * source (Poisson, periodic, k = 0 dropped)
        {
            Launch L(ctx, SGW_PROF_OTHER, 5);
            sgw::launch_real_to_c64(ng * n_samples, source_dev, ctx->B1, st);
            sgw::launch_plane_fwd(n, ctx->B1, Wp, n_samples, ctx->tw, st);
            sgw::launch_pencil(n, Wp, n_samples, 1, kscale, 0.f, ctx->tw, st, 0, nullptr, 0.f,
                               ctx->tune[SGW_TUNE_LINE_FORM]);
            sgw::launch_plane_inv(n, Wp, n_samples, ctx->tw, 2, nullptr, nullptr, nullptr, nullptr, nullptr, 0, vp, st);
            // eta pairs: (eta, d eta = -i v_p eta)
            sgw::launch_kick((int)ng, (const float2*)eta_dev, vp, n_samples, n_eta, psi, st);
            CKL();
        }
        for (int j = 0; j <= n_steps; ++j) {
            // H(t_j): density, Poisson of (rho - rho0) + i d rho, potentials and u^R(t_j)
            {
                Launch L(ctx, SGW_PROF_TDH_DENSITY, 1, (double)ctx->ng * (8.0 * 2 * n_eta * n_samples + 12.0 * n_samples));
                sgw::launch_density_fwd(n, psi, n_samples, n_eta, w, rho0, j == 0 ? 1 : 0, Wp, ctx->tw, st);
            }
            {
                Launch L(ctx, SGW_PROF_OTHER);
                sgw::launch_pencil(n, Wp, n_samples, 1, kscale, 0.f, ctx->tw, st, 0, nullptr, 0.f,
                               ctx->tune[SGW_TUNE_LINE_FORM]);
            }
            {
                Launch L(ctx, SGW_PROF_OTHER);
                sgw::launch_plane_inv(n, Wp, n_samples, ctx->tw, 1, nullptr, ctx->vloc, vtot, dv,
                                      xi ? nullptr : uR_dev + (int64_t)j * ng, uR_stride, nullptr, st);
            }
            if (xi) {
                // U_m(t_j) = <xi_m|u^R(t_j)>, u^R(t_j) = dv: the full-grid u^R is not kept
                Launch L(ctx, SGW_PROF_OTHER, 1, (double)xi->n_xi * xi->K * xi->L * 4.0 * n_samples);
                sgw::launch_xi_project(dv, ng, n_samples, xi->n_xi, xi->K, xi->L, ng, xi->seed, xi->stream, xi->sample0,
                                       (float)(xi->c * ctx->dV), uR_dev + (int64_t)j * xi->n_xi,
                                       (int64_t)(n_steps + 1) * xi->n_xi, st);
            }
            CKL();
            if (j == n_steps) break;
            if (cheb_deg == 0) {
                if (sgw_status s2 = split_step_batch(ctx, psi, B, vtot, dv, dt, F)) return s2;
            } else if (sgw_status s2 = run_series(ctx, plan, psi, psi, B, vtot, dv, ctx->info, j > 0, true, n_samples)) {
                return s2;
            }
        }
        return SGW_OK;
    });
}

sgw_status sgw_tdh_response(sgw_ctx* ctx, const void* eta_dev, const float* source_dev, int n_samples, int n_eta,
                            int n_steps, double dt, int cheb_deg, double weight, float* uR_dev) {
    return tdh_run(ctx, eta_dev, source_dev, n_samples, n_eta, n_steps, dt, cheb_deg, weight, uR_dev, nullptr);
}

sgw_status sgw_tdh_response_xi(sgw_ctx* ctx, const void* eta_dev, const float* source_dev, int n_samples, int n_eta,
                               int n_steps, double dt, int cheb_deg, double weight, uint64_t xi_seed,
                               uint32_t xi_stream, int sample0, int n_xi, double f_g, int L, float* U_dev) {
    sgw_status s = check_ctx(ctx, true);
    if (s) return s;
    XiArgs xa;
    if ((s = xi_args(ctx, xi_seed, xi_stream, sample0, n_xi, f_g, L, &xa))) return s;
    return tdh_run(ctx, eta_dev, source_dev, n_samples, n_eta, n_steps, dt, cheb_deg, weight, U_dev, &xa);
}

sgw_status sgw_time_order(sgw_ctx* ctx, const float* uR_dev, void* u_dev, int n_samples, int n_steps) {
    if (!ctx) return fail(nullptr, SGW_EINVAL, "null context");
    return sgw_time_order_points(ctx, uR_dev, u_dev, n_samples, n_steps, (int)ctx->ng);
}

sgw_status sgw_time_order_points(sgw_ctx* ctx, const float* uR_dev, void* u_dev, int n_samples, int n_steps,
                                 int n_points) {
    sgw_status s = check_ctx(ctx, false);
    if (s) return s;
    if (n_samples < 0 || n_steps < 0 || n_points < 1) return fail(ctx, SGW_EINVAL, "bad time-order arguments");
    if (n_samples == 0) return SGW_OK;
    if (!uR_dev || !u_dev) return fail(ctx, SGW_EINVAL, "null time-order pointers");
    SGW_ALIGNED(ctx, uR_dev, u_dev);
    int M = 4;                                    // the smallest power of two >= 4 (n_steps + 1)
    while (M < 4 * (n_steps + 1)) M *= 2;
    if (M > 4096) return fail(ctx, SGW_EINVAL, "n_steps too large for the time-ordering FFT (M <= 4096)");
    if (ctx->twM_n != M) {
        if (ctx->twM) cudaFree(ctx->twM);
        ctx->twM = nullptr;
        ctx->twM_n = 0;
        CK(cudaMalloc(&ctx->twM, sizeof(float2) * M));
        auto t = twiddles(M);
        CK(cudaMemcpy(ctx->twM, t.data(), sizeof(float2) * M, cudaMemcpyHostToDevice));
        ctx->twM_n = M;
    }
    {
        Launch L(ctx, SGW_PROF_TIME_ORDER, 1, (double)n_points * n_samples * (n_steps + 1) * 12.0);
        sgw::launch_time_order(n_points, uR_dev, (float2*)u_dev, n_samples, n_steps, M, ctx->twM, ctx->stream);
        CKL();
    }
    return SGW_OK;
}

static sgw_status sigma_run(sgw_ctx* ctx, void* zeta_dev, const float* phi_dev, const void* u_dev, int n_samples,
                            int n_steps, double dt, int cheb_deg, int fp64_accum, double* sigma_dev, const XiArgs* xi) {
    sgw_status s = check_ctx(ctx, true);
    if (s) return s;
    if (cheb_deg > 0 && !ctx->have_spectrum) return fail(ctx, SGW_ESTATE, "no spectral interval set");
    if (n_samples < 0 || n_steps < 0 || cheb_deg < 0 || 2 * n_samples > ctx->max_batch)
        return fail(ctx, SGW_EINVAL, "bad sigma arguments (2 n_samples must be <= max_batch)");
    if (n_samples == 0) return SGW_OK;
    if (!zeta_dev || !phi_dev || !u_dev || !sigma_dev) return fail(ctx, SGW_EINVAL, "null sigma pointers");
    SGW_ALIGNED(ctx, zeta_dev, phi_dev, u_dev, sigma_dev);
    cudaStream_t st = ctx->stream;
    const int64_t ng = ctx->ng;
    const int B = 2 * n_samples;
    const int nblk = xi ? (int)std::min<int64_t>((xi->n_xi + 7) / 8, 128) : (int)std::min<int64_t>((ng + 255) / 256, 128);
    void* p;
    if ((s = work(ctx, 4, sizeof(double2) * (size_t)n_samples * (n_steps + 1) * 2 * nblk, &p))) return s;
    double2* partial = (double2*)p;
    std::vector<cd> c[2];
    cd ph[2];
    std::vector<Step> plan;
    const float2* F = nullptr;
    if (cheb_deg > 0) {
        prop_coeffs(ctx, dt, cheb_deg, c, ph);
        plan = clenshaw_plan(c, ph, cheb_deg);
    } else if ((s = split_factors(ctx, dt, &F))) {
        return s;
    }
    std::vector<sgw::VecInfo> info(B);
    for (int sm = 0; sm < n_samples; ++sm) {
        info[2 * sm] = sgw::VecInfo{0, -1, -1, 1};      // zeta_occ: backwards, e^{+i H t}
        info[2 * sm + 1] = sgw::VecInfo{0, -1, -1, 0};  // zeta_unocc: forwards
    }
    if ((s = upload_info(ctx, info))) return s;
    float2* z = (float2*)zeta_dev;
    const int64_t u_ss = (int64_t)(n_steps + 1) * (xi ? xi->n_xi : ng);
    std::vector<uint64_t> key = {4, (uint64_t)n_samples, (uint64_t)n_steps, bits(dt), (uint64_t)cheb_deg,
                                 (uint64_t)fp64_accum, (uint64_t)zeta_dev, (uint64_t)phi_dev, (uint64_t)u_dev,
                                 (uint64_t)sigma_dev, (uint64_t)partial};
    if (xi) {
        key.insert(key.end(), {xi->seed, (uint64_t)xi->stream, (uint64_t)xi->sample0, (uint64_t)xi->n_xi,
                               (uint64_t)xi->K, (uint64_t)xi->L});
    }
    return graphed(ctx, key, [&]() -> sgw_status {
    for (int j = 0; j <= n_steps; ++j) {
        {
            if (xi) {
                Launch L(ctx, SGW_PROF_SIGMA, 1,
                         (double)xi->n_xi * xi->K * xi->L * n_samples * (8.0 * 2 + 4.0) + 8.0 * xi->n_xi * n_samples);
                sgw::launch_sigma_accum_xi(z, phi_dev, (const float2*)u_dev, n_samples, u_ss, j, n_steps, xi->n_xi,
                                           xi->K, xi->L, ng, xi->seed, xi->stream, xi->sample0, (float)xi->c, fp64_accum,
                                           partial, nblk, st);
            } else {
                Launch L(ctx, SGW_PROF_SIGMA, 1, (double)ng * n_samples * (8.0 * 3 + 4.0));
                sgw::launch_sigma_accum((int)ng, z, phi_dev, (const float2*)u_dev, n_samples, u_ss, j, n_steps,
                                        (float)ctx->dV, fp64_accum, partial, nblk, st);
            }
            CKL();
        }
        if (j == n_steps) break;
        if (cheb_deg == 0) {
            if (sgw_status s2 = split_step_batch(ctx, z, B, ctx->vloc, nullptr, dt, F)) return s2;
        } else if (sgw_status s2 = run_series(ctx, plan, z, z, B, ctx->vloc, nullptr, ctx->info, j > 0,
                                               j + 1 < n_steps)) {
            return s2;
        }
    }
    {
        Launch L(ctx, SGW_PROF_OTHER);
        sgw::launch_sigma_reduce(partial, n_samples, n_steps, nblk, ctx->dV, fp64_accum, sigma_dev, st);
        CKL();
    }
    return SGW_OK;
    });
}

sgw_status sgw_sigma_c(sgw_ctx* ctx, void* zeta_dev, const float* phi_dev, const void* u_dev, int n_samples, int n_steps,
                       double dt, int cheb_deg, int fp64_accum, double* sigma_dev) {
    return sigma_run(ctx, zeta_dev, phi_dev, u_dev, n_samples, n_steps, dt, cheb_deg, fp64_accum, sigma_dev, nullptr);
}

sgw_status sgw_sigma_c_xi(sgw_ctx* ctx, void* zeta_dev, const float* phi_dev, const void* u_dev, int n_samples,
                          int n_steps, double dt, int cheb_deg, int fp64_accum, uint64_t xi_seed, uint32_t xi_stream,
                          int sample0, int n_xi, double f_g, int L, double* sigma_dev) {
    sgw_status s = check_ctx(ctx, true);
    if (s) return s;
    XiArgs xa;
    if ((s = xi_args(ctx, xi_seed, xi_stream, sample0, n_xi, f_g, L, &xa))) return s;
    return sigma_run(ctx, zeta_dev, phi_dev, u_dev, n_samples, n_steps, dt, cheb_deg, fp64_accum, sigma_dev, &xa);
}

sgw_status sgw_exchange(sgw_ctx* ctx, const void* eta_dev, const float* phi_dev, int n_samples, int n_eta,
                        double* x_dev) {
    sgw_status s = check_ctx(ctx, false);
    if (s) return s;
    if (n_samples < 0 || n_eta < 1 || n_eta > ctx->max_batch) return fail(ctx, SGW_EINVAL, "bad exchange arguments");
    if (n_samples == 0) return SGW_OK;
    if (!eta_dev || !phi_dev || !x_dev) return fail(ctx, SGW_EINVAL, "null exchange pointers");
    SGW_ALIGNED(ctx, eta_dev, phi_dev);
    cudaStream_t st = ctx->stream;
    const int64_t ng = ctx->ng;
    const float kscale = (float)std::pow(2.0 * M_PI / ctx->L, 2);
    const int per_call = std::max(1, ctx->max_batch / n_eta);
    void* wp;
    if ((s = work(ctx, 10, sizeof(double) * (size_t)sgw::pencil_blocks(ctx->n) * per_call * n_eta, &wp))) return s;
    for (int s0 = 0; s0 < n_samples; s0 += per_call) {
        const int ns = std::min(per_call, n_samples - s0);
        const int B = ns * n_eta;
        Launch L(ctx, SGW_PROF_OTHER, 4);
        sgw::launch_scale_mul((int64_t)B * ng, phi_dev, (int)ng, (const float2*)eta_dev + (size_t)s0 * n_eta * ng,
                              ctx->B1, st);
        sgw::launch_plane_fwd(ctx->n, ctx->B1, ctx->W, B, ctx->tw, st);
        // <f|v_C f> = (dV / N) sum_k 4 pi/k^2 |F(k)|^2 ; X = -(1/n_eta) sum_l
        sgw::launch_pencil_coulomb_energy(ctx->n, ctx->W, B, n_eta, kscale, -ctx->dV / (double)ng / n_eta, ctx->tw,
                                          (double*)wp, x_dev + s0, st);
        CKL();
    }
    return SGW_OK;
}

sgw_status sgw_sigma_omega(sgw_ctx* ctx, const double* sigma_dev, int n_samples, int n_steps, double dt, double gamma,
                           const double* omega_dev, int n_omega, int fp64, double* out_dev) {
    sgw_status s = check_ctx(ctx, false);
    if (s) return s;
    if (n_samples < 1 || n_steps < 0 || n_omega < 0 || !sigma_dev || (!omega_dev && n_omega) || (!out_dev && n_omega))
        return fail(ctx, SGW_EINVAL, "bad sigma-omega arguments");
    sgw::launch_sigma_omega(sigma_dev, n_samples, n_steps, dt, gamma, omega_dev, n_omega, fp64, out_dev, ctx->stream);
    CKL();
    return SGW_OK;
}

sgw_status sgw_qp_energy(sgw_ctx* ctx, const double* sigma_dev, const double* x_dev, int n_samples, int n_steps,
                         double dt, double gamma, double eps_ks, double vxc, double window, double step, int fp64,
                         double* result_host) {
    sgw_status s = check_ctx(ctx, false);
    if (s) return s;
    if (n_samples < 1 || n_steps < 0 || !(window > 0) || !(step > 0) || !sigma_dev || !x_dev || !result_host)
        return fail(ctx, SGW_EINVAL, "bad QP arguments");
    const double r = 2.0 * window / step;
    if (!std::isfinite(r) || r + 1.0 > 1e8) return fail(ctx, SGW_EINVAL, "QP scan of 2 window/step + 1 > 1e8 points");
    const int n_scan = (int)std::llround(r) + 1;
    void* p;
    const size_t bytes = sizeof(double) * (((n_scan + 1) & ~1) + 2 * (2 * n_steps + 1)) + 4 * sizeof(double);
    if ((s = work(ctx, 5, bytes, &p))) return s;
    double* scan = (double*)p;
    double* result = ctx->scal + 16;
    {
        Launch L(ctx, SGW_PROF_OTHER, 3);
        sgw::launch_qp(sigma_dev, x_dev, n_samples, n_steps, dt, gamma, eps_ks, vxc, window, step, fp64, scan, n_scan,
                       result, ctx->stream);
        CKL();
    }
    CK(cudaMemcpyAsync(result_host, result, 4 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (std::isnan(result_host[0])) return fail(ctx, SGW_ENOCONV, "no sign change of the QP equation in the window");
    return SGW_OK;
}

// Wave vectors m, 0 < |m|^2 <= m2max, one of each +-m pair (first non-zero component > 0),
// ordered by |m|^2 and then lexicographically (mx, my, mz).
static std::vector<int4> cv_kset(int m2max) {
    std::vector<int4> ks;
    const int r = (int)std::floor(std::sqrt((double)m2max));
    for (int a = -r; a <= r; ++a)
        for (int b = -r; b <= r; ++b)
            for (int c = -r; c <= r; ++c) {
                const int n2 = a * a + b * b + c * c;
                if (n2 == 0 || n2 > m2max) continue;
                const int first = a != 0 ? a : (b != 0 ? b : c);
                if (first > 0) ks.push_back(make_int4(a, b, c, n2));
            }
    std::sort(ks.begin(), ks.end(), [](const int4& p, const int4& q) {
        if (p.w != q.w) return p.w < q.w;
        if (p.x != q.x) return p.x < q.x;
        if (p.y != q.y) return p.y < q.y;
        return p.z < q.z;
    });
    return ks;
}

int sgw_cv_feature_count(int m2max) { return m2max < 1 ? 2 : 2 * ((int)cv_kset(m2max).size() + 1); }

sgw_status sgw_cv_features(sgw_ctx* ctx, const void* noise_dev, int n_samples, int n_vec, const float* phi_dev,
                           int m2max, float* feat_dev) {
    sgw_status s = check_ctx(ctx, false);
    if (s) return s;
    if (n_samples < 0 || n_vec < 1 || m2max < 1) return fail(ctx, SGW_EINVAL, "bad feature arguments");
    if (n_samples == 0) return SGW_OK;
    if (!noise_dev || !phi_dev || !feat_dev) return fail(ctx, SGW_EINVAL, "null feature pointers");
    SGW_ALIGNED(ctx, noise_dev, phi_dev);
    const std::vector<int4> ks = cv_kset(m2max);
    const int nk = (int)ks.size();
    const int chunk = std::max(1, ctx->max_batch / n_vec);
    if (n_vec > ctx->max_batch) return fail(ctx, SGW_EINVAL, "n_vec must not exceed max_batch");
    void *p, *q;
    if ((s = work(ctx, 6, sizeof(int4) * nk, &p))) return s;
    if ((s = work(ctx, 7, sizeof(float) * (size_t)chunk * n_vec * (2 * nk + 1), &q))) return s;
    int4* ksd = (int4*)p;
    float* raw = (float*)q;
    CK(cudaMemcpyAsync(ksd, ks.data(), sizeof(int4) * nk, cudaMemcpyHostToDevice, ctx->stream));
    const float kscale = (float)std::pow(2.0 * M_PI / ctx->L, 2);
    for (int s0 = 0; s0 < n_samples; s0 += chunk) {
        const int ns = std::min(chunk, n_samples - s0);
        const int nvv = ns * n_vec;
        Launch L(ctx, SGW_PROF_OTHER, 4);
        sgw::launch_cv_source(ctx->ng, (const float2*)noise_dev + (size_t)s0 * n_vec * ctx->ng, ctx->ng, phi_dev, nvv,
                              ctx->B1, ctx->stream);
        sgw::launch_plane_fwd(ctx->n, ctx->B1, ctx->W, nvv, ctx->tw, ctx->stream);
        sgw::launch_cv_gather(ctx->n, ctx->W, nvv, nk, ksd, kscale, (float)ctx->dV, ctx->tw, raw, ctx->stream);
        sgw::launch_cv_combine(ns, n_vec, nk, raw, feat_dev + (size_t)s0 * 2 * (nk + 1), ctx->stream);
        CKL();
    }
    // the host list must outlive the (pageable, stream-ordered) copy
    CK(cudaStreamSynchronize(ctx->stream));
    return SGW_OK;
}

sgw_status sgw_cv_standardize(sgw_ctx* ctx, const double* y_dev, int n_rows, int n_out, int compute_stats,
                              double* mu_dev, double* sd_dev, float* t_dev) {
    sgw_status s = check_ctx(ctx, false);
    if (s) return s;
    if (n_rows < 1 || n_out < 1 || !y_dev || !mu_dev || !sd_dev || !t_dev)
        return fail(ctx, SGW_EINVAL, "bad standardize arguments");
    Launch L(ctx, SGW_PROF_OTHER, 2);
    if (compute_stats) sgw::launch_cv_stats(n_rows, n_out, y_dev, mu_dev, sd_dev, ctx->stream);
    sgw::launch_cv_standardize((int64_t)n_rows * n_out, n_out, y_dev, mu_dev, sd_dev, t_dev, ctx->stream);
    CKL();
    return SGW_OK;
}

sgw_status sgw_cv_standardize_f32(sgw_ctx* ctx, float* x_dev, int n_rows, int n_cols, int compute_stats,
                                  double* mu_dev, double* sd_dev) {
    sgw_status s = check_ctx(ctx, false);
    if (s) return s;
    if (n_rows < 1 || n_cols < 1 || !x_dev || !mu_dev || !sd_dev)
        return fail(ctx, SGW_EINVAL, "bad standardize arguments");
    Launch L(ctx, SGW_PROF_OTHER, 2);
    sgw::launch_cv_standardize_f32(n_rows, n_cols, x_dev, mu_dev, sd_dev, compute_stats, ctx->stream);
    CKL();
    return SGW_OK;
}

sgw_status sgw_cv_rows(sgw_ctx* ctx, const float* f_cheap_dev, int n_cheap, const float* f_paired_dev,
                       const double* y_paired_dev, int n_paired, int n_out, const double* mu_dev,
                       const double* sd_dev, double* rows_dev) {
    sgw_status s = check_ctx(ctx, false);
    if (s) return s;
    if (n_cheap < 0 || n_paired < 1 || n_out < 1 || !y_paired_dev || !rows_dev ||
        (n_cheap > 0 && (!f_cheap_dev || !f_paired_dev || !mu_dev || !sd_dev)))
        return fail(ctx, SGW_EINVAL, "bad control-variate arguments");
    Launch L(ctx, SGW_PROF_OTHER);
    sgw::launch_cv_rows(n_cheap, n_paired, n_out, f_cheap_dev, f_paired_dev, y_paired_dev, mu_dev, sd_dev, rows_dev,
                        ctx->stream);
    CKL();
    return SGW_OK;
}

// ---------------------------------------------------------------- control variate: linear part
static std::vector<int> cv_shell_of_k(int m2max, int* n_shells) {
    const std::vector<int4> ks = cv_kset(m2max);
    std::vector<int> sq;
    for (const int4& k : ks)
        if (sq.empty() || sq.back() != k.w) sq.push_back(k.w);     // ks is sorted by |m|^2
    std::vector<int> idx(ks.size());
    for (size_t i = 0; i < ks.size(); ++i)
        idx[i] = (int)(std::lower_bound(sq.begin(), sq.end(), ks[i].w) - sq.begin());
    *n_shells = (int)sq.size();
    return idx;
}

int sgw_cv_shell_count(int m2max) {
    if (m2max < 1) return 2;
    int ns = 0;
    cv_shell_of_k(m2max, &ns);
    return 2 * (ns + 1);
}

sgw_status sgw_cv_shell_sums(sgw_ctx* ctx, const float* feat_dev, int n_samples, int m2max, float* out_dev) {
    sgw_status s = check_ctx(ctx, false);
    if (s) return s;
    if (n_samples < 0 || m2max < 1) return fail(ctx, SGW_EINVAL, "bad shell-sum arguments");
    if (n_samples == 0) return SGW_OK;
    if (!feat_dev || !out_dev) return fail(ctx, SGW_EINVAL, "null shell-sum pointers");
    int ns = 0;
    const std::vector<int> idx = cv_shell_of_k(m2max, &ns);
    void* p;
    if ((s = work(ctx, 9, sizeof(int) * idx.size(), &p))) return s;
    CK(cudaMemcpyAsync(p, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));       // idx is a host temporary
    Launch L(ctx, SGW_PROF_OTHER);
    sgw::launch_cv_shells(n_samples, (int)idx.size(), ns, (const int*)p, feat_dev, out_dev, ctx->stream);
    CKL();
    return SGW_OK;
}

int64_t sgw_cv_linear_size(int p, int o) { return (p < 1 || o < 1) ? 0 : 2 * (int64_t)p + o + (int64_t)p * o; }

sgw_status sgw_cv_linear_fit(sgw_ctx* ctx, const float* x_dev, const double* y_dev, int n, int p, int o, double ridge,
                             double* model_dev) {
    sgw_status s = check_ctx(ctx, false);
    if (s) return s;
    if (n < 2 || p < 1 || p > 256 || o < 1 || !(ridge >= 0.0) || !x_dev || !y_dev || !model_dev)
        return fail(ctx, SGW_EINVAL, "bad linear-fit arguments");
    // work: x in FP64 [n][p], sd of y [o], G [p][p], C [p][o]
    const size_t nx = (size_t)n * p, ng = (size_t)p * p, nc = (size_t)p * o;
    void* w;
    if ((s = work(ctx, 8, sizeof(double) * (nx + o + ng + nc), &w))) return s;
    double* xd = (double*)w;
    double* sdy = xd + nx;
    double* G = sdy + o;
    double* C = G + ng;
    double* mu = model_dev;
    double* sd = model_dev + p;
    double* ybar = model_dev + 2 * p;
    double* B = model_dev + 2 * p + o;
    {
        Launch L(ctx, SGW_PROF_OTHER, 5);
        sgw::launch_f32_to_f64((int64_t)nx, x_dev, xd, ctx->stream);
        sgw::launch_cv_stats(n, p, xd, mu, sd, ctx->stream);
        sgw::launch_cv_stats(n, o, y_dev, ybar, sdy, ctx->stream);
        sgw::launch_cv_gram(n, p, xd, mu, sd, G, ctx->stream);
        sgw::launch_cv_xty(n, p, o, xd, mu, sd, y_dev, ybar, C, ctx->stream);
        CKL();
    }
    // (G + ridge n I) B = C by Cholesky on the host, in FP64
    std::vector<double> g(ng), c(nc);
    CK(cudaMemcpyAsync(g.data(), G, sizeof(double) * ng, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(c.data(), C, sizeof(double) * nc, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int a = 0; a < p; ++a) g[(size_t)a * p + a] += ridge * n;
    for (int j = 0; j < p; ++j) {
        double d = g[(size_t)j * p + j];
        for (int k = 0; k < j; ++k) d -= g[(size_t)j * p + k] * g[(size_t)j * p + k];
        if (!(d > 0.0)) return fail(ctx, SGW_ENOCONV, "linear fit: normal matrix is not positive definite");
        const double ljj = std::sqrt(d);
        g[(size_t)j * p + j] = ljj;
        for (int i = j + 1; i < p; ++i) {
            double v = g[(size_t)i * p + j];
            for (int k = 0; k < j; ++k) v -= g[(size_t)i * p + k] * g[(size_t)j * p + k];
            g[(size_t)i * p + j] = v / ljj;
        }
    }
    for (int col = 0; col < o; ++col) {
        std::vector<double> z(p);
        for (int i = 0; i < p; ++i) {
            double v = c[(size_t)i * o + col];
            for (int k = 0; k < i; ++k) v -= g[(size_t)i * p + k] * z[k];
            z[i] = v / g[(size_t)i * p + i];
        }
        for (int i = p - 1; i >= 0; --i) {
            double v = z[i];
            for (int k = i + 1; k < p; ++k) v -= g[(size_t)k * p + i] * c[(size_t)k * o + col];
            c[(size_t)i * o + col] = v / g[(size_t)i * p + i];
        }
    }
    CK(cudaMemcpyAsync(B, c.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return SGW_OK;
}

sgw_status sgw_cv_linear_apply(sgw_ctx* ctx, const double* model_dev, const float* x_dev, int n, int p, int o,
                               const double* y_dev, double* out_dev) {
    sgw_status s = check_ctx(ctx, false);
    if (s) return s;
    if (n < 0 || p < 1 || o < 1 || !model_dev || (n > 0 && (!x_dev || !out_dev)))
        return fail(ctx, SGW_EINVAL, "bad linear-apply arguments");
    Launch L(ctx, SGW_PROF_OTHER);
    sgw::launch_cv_lin_apply(n, p, o, model_dev, x_dev, y_dev, out_dev, ctx->stream);
    CKL();
    return SGW_OK;
}

sgw_status sgw_cv_linear_rows(sgw_ctx* ctx, const double* model_dev, const float* x_cheap_dev, int n_cheap,
                              const float* x_paired_dev, int n_paired, int p, int o, const double* y_dev,
                              double* y_out_dev) {
    sgw_status s = check_ctx(ctx, false);
    if (s) return s;
    if (n_cheap < 1 || n_paired < 1 || p < 1 || o < 1 || !model_dev || !x_cheap_dev || !x_paired_dev || !y_dev ||
        !y_out_dev)
        return fail(ctx, SGW_EINVAL, "bad linear-rows arguments");
    void* w;
    if ((s = work(ctx, 9, sizeof(double) * std::max(p, 64), &w))) return s;
    Launch L(ctx, SGW_PROF_OTHER, 2);
    sgw::launch_cv_lin_rows(n_cheap, n_paired, p, o, model_dev, x_cheap_dev, x_paired_dev, y_dev, (double*)w,
                            y_out_dev, ctx->stream);
    CKL();
    return SGW_OK;
}

sgw_status sgw_profile(sgw_ctx* ctx, int enable) {
    sgw_status s = check_ctx(ctx, false);
    if (s) return s;
    prof_flush(ctx);
    for (int k = 0; k < SGW_PROF_KINDS; ++k) {
        ctx->prof_ms[k] = 0;
        ctx->prof_n[k] = 0;
        ctx->prof_bytes[k] = 0;
    }
    ctx->prof = enable != 0;
    return SGW_OK;
}

sgw_status sgw_profile_read(sgw_ctx* ctx, int kind, double* total_ms_host, int64_t* count_host,
                            double* alg_bytes_host) {
    sgw_status s = check_ctx(ctx, false);
    if (s) return s;
    if (kind < 0 || kind >= SGW_PROF_KINDS || !total_ms_host || !count_host)
        return fail(ctx, SGW_EINVAL, "bad profile kind");
    prof_flush(ctx);
    *total_ms_host = ctx->prof_ms[kind];
    *count_host = ctx->prof_n[kind];
    if (alg_bytes_host) *alg_bytes_host = ctx->prof_bytes[kind];
    return SGW_OK;
}

sgw_status sgw_launch_count(sgw_ctx* ctx, int64_t* count_host) {
    if (!ctx || !count_host) return fail(ctx, SGW_EINVAL, "null argument");
    *count_host = ctx->launches;
    return SGW_OK;
}

}  // extern "C"
