// Runtime services around the hot path: stream synchronisation with kernel
// error reporting, the RWG -> (group, slot) table, plan checkpoints, CUDA-graph
// capture of the two stages, and the autotuner that picks launch shapes, queue
// orders and the multi-RHS engine by timing them on the plan's own data.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "internal.h"

struct tfmm_graph {
    tfmm_plan* plan = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace tfmm {
namespace {

// ------------------------------------------------------------- checkpoints
// File layout (native little-endian, every field back to back):
//   char[8] "TFMMPLAN", uint32 version, uint32 flags (bit 0: geometry, bit 1: grid),
//   uint32 sizeof(tfmm_params), tfmm_params,
//   int32 L, n_theta, n_phi, G, K[3]; int64 N; double k, w_phi, setup_ms[4],
//   double theta[n_theta], w_theta[n_theta], phi[n_phi]; float weights[n_dir],
//   int64 grp_off[G+1], grp_rwg[N]; double centres[3G]; int32 ranks[6G],
//   RwgGeom geom[N] (flag bit 0),
//   per (g, alpha): complex128 U_theta (n_theta x r_theta), U_phi, U_beta, core
//   (column-major, as tfmm_plan_export_factors), then char[8] "TFMMEND."
constexpr char kMagic[8] = {'T', 'F', 'M', 'M', 'P', 'L', 'A', 'N'};
constexpr char kTrailer[8] = {'T', 'F', 'M', 'M', 'E', 'N', 'D', '.'};
constexpr uint32_t kVersion = 1;

struct File {
    FILE* f = nullptr;
    std::string path;
    File(const char* p, const char* mode) : f(std::fopen(p, mode)), path(p) {
        if (!f) fail(TFMM_IO, "cannot open " + path);
    }
    ~File() {
        if (f) std::fclose(f);
    }
    void put(const void* d, size_t n) {
        if (n && std::fwrite(d, 1, n, f) != n) fail(TFMM_IO, "write failed: " + path);
    }
    void get(void* d, size_t n) {
        if (n && std::fread(d, 1, n, f) != n) fail(TFMM_IO, "truncated checkpoint: " + path);
    }
    template <class T>
    void put_v(const std::vector<T>& v) { put(v.data(), sizeof(T) * v.size()); }
    template <class T>
    void get_v(std::vector<T>& v, size_t n) {
        v.resize(n);
        get(v.data(), sizeof(T) * n);
    }
    void close() {
        FILE* g = f;
        f = nullptr;
        if (std::fclose(g) != 0) fail(TFMM_IO, "close failed: " + path);
    }
};

int64_t item_elems(const Plan& P, int g, int rt, int rp, int rb) {
    const int64_t nb = P.grp_off[g + 1] - P.grp_off[g];
    return (int64_t)P.n_theta * rt + (int64_t)P.n_phi * rp + nb * rb + (int64_t)rt * rp * rb;
}

void save_plan(const Plan& P, const char* path) {
    File F(path, "wb");
    F.put(kMagic, 8);
    const uint32_t flags = (P.has_geometry ? 1u : 0u) | (P.theta.empty() ? 0u : 2u);
    const uint32_t head[3] = {kVersion, flags, (uint32_t)sizeof(tfmm_params)};
    F.put(head, sizeof(head));
    F.put(&P.params, sizeof(tfmm_params));
    const int32_t dims[7] = {P.L, P.n_theta, P.n_phi, P.G, P.K[0], P.K[1], P.K[2]};
    F.put(dims, sizeof(dims));
    F.put(&P.N, sizeof(int64_t));
    const double sc[6] = {P.k, P.w_phi, P.setup_ms[0], P.setup_ms[1], P.setup_ms[2], P.setup_ms[3]};
    F.put(sc, sizeof(sc));
    std::vector<double> th(P.n_theta, 0.0), wt(P.n_theta, 0.0), ph(P.n_phi, 0.0);
    if (!P.theta.empty()) { th = P.theta; wt = P.w_theta; ph = P.phi; }
    F.put_v(th); F.put_v(wt); F.put_v(ph);
    F.put_v(P.weights);
    F.put_v(P.grp_off);
    F.put_v(P.grp_rwg);
    std::vector<double> cen(P.centres);
    cen.resize((size_t)3 * P.G, 0.0);
    F.put_v(cen);
    F.put_v(P.ranks);
    if (P.has_geometry) F.put_v(P.geom);
    std::vector<double2> buf;
    for (int g = 0; g < P.G; ++g)
        for (int al = 0; al < 2; ++al) {
            const HostFactors64& h = P.f64[(size_t)g * 2 + al];
            buf.resize(item_elems(P, g, h.rt, h.rp, h.rb));
            TFMM_CUDA_CHECK(cudaMemcpy(buf.data(), h.base, sizeof(double2) * buf.size(), cudaMemcpyDeviceToHost));
            F.put_v(buf);
        }
    F.put(kTrailer, 8);
    F.close();
}

std::unique_ptr<tfmm_plan> load_plan(const char* path, cudaStream_t s) {
    File F(path, "rb");
    char magic[8];
    F.get(magic, 8);
    if (std::memcmp(magic, kMagic, 8) != 0) fail(TFMM_IO, "not a tfmm plan checkpoint: " + F.path);
    uint32_t head[3];
    F.get(head, sizeof(head));
    if (head[0] != kVersion) fail(TFMM_IO, "unsupported checkpoint version " + std::to_string(head[0]));
    if (head[2] != sizeof(tfmm_params)) fail(TFMM_IO, "checkpoint written by an incompatible build");
    auto h = std::make_unique<tfmm_plan>();
    Plan& P = h->p;
    F.get(&P.params, sizeof(tfmm_params));
    P.params.keep_dense = 0;  // dense tensors are not checkpointed
    int32_t dims[7];
    F.get(dims, sizeof(dims));
    P.L = dims[0]; P.n_theta = dims[1]; P.n_phi = dims[2]; P.G = dims[3];
    P.K[0] = dims[4]; P.K[1] = dims[5]; P.K[2] = dims[6];
    F.get(&P.N, sizeof(int64_t));
    auto bad = [&](bool c, const char* what) {
        if (c) fail(TFMM_IO, std::string("corrupt checkpoint (") + what + "): " + F.path);
    };
    bad(P.n_theta < 1 || P.n_theta > 4096 || P.n_phi < 1 || P.n_phi > 8192, "grid");
    bad(P.G < 1 || P.G > (1 << 26) || P.N < 1 || P.N >= ((int64_t)1 << 31), "sizes");
    bad(P.params.max_rhs < 1, "params");
    P.n_dir = P.n_theta * P.n_phi;
    P.ld_dir = (int)round_up(P.n_dir, 2);
    {
        // the arrays the header announces must fit in what is left of the file (no
        // allocation sized by a corrupt header)
        const long here = std::ftell(F.f);
        std::fseek(F.f, 0, SEEK_END);
        const long end = std::ftell(F.f);
        std::fseek(F.f, here, SEEK_SET);
        const double need = 6.0 * 8 + (2.0 * P.n_theta + P.n_phi) * 8 + 4.0 * P.n_dir + 8.0 * (P.G + 1) +
                            8.0 * P.N + 24.0 * P.G + 24.0 * P.G + ((head[1] & 1u) ? (double)sizeof(RwgGeom) * P.N : 0.0) +
                            8;
        bad(here < 0 || end < 0 || (double)(end - here) < need, "file shorter than its header announces");
    }
    double sc[6];
    F.get(sc, sizeof(sc));
    P.k = sc[0]; P.w_phi = sc[1];
    for (int i = 0; i < 4; ++i) P.setup_ms[i] = sc[2 + i];
    F.get_v(P.theta, P.n_theta);
    F.get_v(P.w_theta, P.n_theta);
    F.get_v(P.phi, P.n_phi);
    if (!(head[1] & 2u)) {  // plan made from factors: no quadrature rule
        P.theta.clear(); P.w_theta.clear(); P.phi.clear();
    }
    F.get_v(P.weights, P.n_dir);
    F.get_v(P.grp_off, (size_t)P.G + 1);
    bad(P.grp_off[0] != 0 || P.grp_off[P.G] != P.N, "group offsets");
    for (int g = 0; g < P.G; ++g) bad(P.grp_off[g + 1] <= P.grp_off[g], "group offsets");
    F.get_v(P.grp_rwg, (size_t)P.N);
    {
        std::vector<char> seen(P.N, 0);
        for (int64_t v : P.grp_rwg) {
            bad(v < 0 || v >= P.N || seen[v], "group members");
            seen[v] = 1;
        }
    }
    F.get_v(P.centres, (size_t)3 * P.G);
    F.get_v(P.ranks, (size_t)6 * P.G);
    for (int g = 0; g < P.G; ++g)
        for (int al = 0; al < 2; ++al) {
            const int* rk = &P.ranks[((size_t)g * 2 + al) * 3];
            const int64_t nb = P.grp_off[g + 1] - P.grp_off[g];
            bad(rk[0] < 1 || rk[0] > P.n_theta || rk[1] < 1 || rk[1] > P.n_phi || rk[2] < 1 || rk[2] > nb, "ranks");
        }
    P.has_geometry = (head[1] & 1u) != 0;
    if (P.has_geometry) F.get_v(P.geom, (size_t)P.N);
    // factors: one device arena, filled item by item
    int64_t total = 0;
    for (int g = 0; g < P.G; ++g)
        for (int al = 0; al < 2; ++al) {
            const int* rk = &P.ranks[((size_t)g * 2 + al) * 3];
            total += item_elems(P, g, rk[0], rk[1], rk[2]);
        }
    upload_common(P, s);
    double2* arena = nullptr;
    TFMM_CUDA_CHECK(device_malloc(&arena, sizeof(double2) * total));
    P.f64_arenas.push_back(arena);
    P.f64.assign((size_t)P.G * 2, HostFactors64{});
    std::vector<double2> buf;
    int64_t pos = 0;
    for (int g = 0; g < P.G; ++g)
        for (int al = 0; al < 2; ++al) {
            const int* rk = &P.ranks[((size_t)g * 2 + al) * 3];
            HostFactors64& hf = P.f64[(size_t)g * 2 + al];
            hf.rt = rk[0]; hf.rp = rk[1]; hf.rb = rk[2];
            hf.base = arena + pos;
            const int64_t n = item_elems(P, g, rk[0], rk[1], rk[2]);
            F.get_v(buf, n);
            for (const double2& v : buf) bad(!std::isfinite(v.x) || !std::isfinite(v.y), "non-finite factor");
            TFMM_CUDA_CHECK(cudaMemcpy(hf.base, buf.data(), sizeof(double2) * n, cudaMemcpyHostToDevice));
            pos += n;
        }
    char tail[8];
    F.get(tail, 8);
    bad(std::memcmp(tail, kTrailer, 8) != 0, "trailer");
    if (std::fgetc(F.f) != EOF) fail(TFMM_IO, "trailing bytes after the checkpoint: " + F.path);
    if (P.has_geometry) {
        TFMM_CUDA_CHECK(device_malloc(&P.d_geom, sizeof(RwgGeom) * P.N));
        TFMM_CUDA_CHECK(cudaMemcpyAsync(P.d_geom, P.geom.data(), sizeof(RwgGeom) * P.N, cudaMemcpyHostToDevice, s));
    }
    pack_factors_fp32(P, s);
    TFMM_CUDA_CHECK(cudaStreamSynchronize(s));
    return h;
}

// ------------------------------------------------------------------- graphs
void run_stages(tfmm_plan* plan, int stages, const tfmm_cfloat* x, int R, int64_t ldx, tfmm_cfloat* spectra,
                int weights, tfmm_cfloat beta, tfmm_cfloat* y, int64_t ldy, cudaStream_t s) {
    if (stages & 1)
        if (tfmm_aggregate(plan, x, R, ldx, spectra, s) != TFMM_OK) fail(TFMM_CUDA, last_error());
    if (stages & 2)
        if (tfmm_disaggregate(plan, spectra, R, weights, beta, y, ldy, s) != TFMM_OK) fail(TFMM_CUDA, last_error());
}

struct StreamGuard {
    cudaStream_t s = nullptr;
    StreamGuard() { TFMM_CUDA_CHECK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)); }
    ~StreamGuard() {
        if (s) cudaStreamDestroy(s);
    }
};

// ---------------------------------------------------------------- autotuner
struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    Timer() {
        TFMM_CUDA_CHECK(cudaEventCreate(&a));
        TFMM_CUDA_CHECK(cudaEventCreate(&b));
    }
    ~Timer() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};

struct Scratch {
    DeviceBuffer x, spec, y;
};

// mean ms of `reps` back-to-back launches of f after one untimed launch
template <class Fn>
double time_ms(Fn&& f, int reps, cudaStream_t s, Timer& t) {
    f();
    TFMM_CUDA_CHECK(cudaEventRecord(t.a, s));
    for (int i = 0; i < reps; ++i) f();
    TFMM_CUDA_CHECK(cudaEventRecord(t.b, s));
    TFMM_CUDA_CHECK(cudaEventSynchronize(t.b));
    float ms = 0.f;
    TFMM_CUDA_CHECK(cudaEventElapsedTime(&ms, t.a, t.b));
    return (double)ms / reps;
}

}  // namespace
}  // namespace tfmm

using namespace tfmm;

extern "C" {

tfmm_status tfmm_sync(tfmm_plan* plan, void* stream) {
    return guarded([&] {
        TFMM_REQUIRE(plan, "null plan");
        TFMM_CUDA_CHECK(cudaStreamSynchronize((cudaStream_t)stream));
        int errs = 0;
        if (plan->p.tc_err.p)
            TFMM_CUDA_CHECK(cudaMemcpy(&errs, plan->p.tc_err.p, sizeof(int), cudaMemcpyDeviceToHost));
        if (errs) fail(TFMM_CUDA, std::to_string(errs) + " tensor-core tile(s) gave up waiting; their outputs are invalid");
    });
}

tfmm_status tfmm_plan_rwg_perm(const tfmm_plan* plan, int32_t* group, int32_t* slot) {
    return guarded([&] {
        TFMM_REQUIRE(plan && group && slot, "null argument");
        const Plan& P = plan->p;
        for (int g = 0; g < P.G; ++g)
            for (int64_t q = P.grp_off[g]; q < P.grp_off[g + 1]; ++q) {
                group[P.grp_rwg[q]] = g;
                slot[P.grp_rwg[q]] = (int32_t)(q - P.grp_off[g]);
            }
    });
}

tfmm_status tfmm_plan_save(const tfmm_plan* plan, const char* path) {
    return guarded([&] {
        TFMM_REQUIRE(plan && path, "null argument");
        save_plan(plan->p, path);
    });
}

tfmm_status tfmm_plan_load(const char* path, void* stream, tfmm_plan** out) {
    return guarded([&] {
        TFMM_REQUIRE(out && path, "null argument");
        *out = nullptr;
        *out = load_plan(path, (cudaStream_t)stream).release();
    });
}

tfmm_status tfmm_graph_capture(tfmm_plan* plan, int32_t stages, const tfmm_cfloat* x, int32_t R, int64_t ldx,
                               tfmm_cfloat* spectra, int32_t apply_weights, tfmm_cfloat beta, tfmm_cfloat* y,
                               int64_t ldy, tfmm_graph** out) {
    return guarded([&] {
        TFMM_REQUIRE(out, "null output");
        *out = nullptr;
        TFMM_REQUIRE(plan, "null plan");
        TFMM_REQUIRE(stages >= 1 && stages <= 3, "stages must be 1 (aggregate), 2 (disaggregate) or 3 (both)");
        TFMM_REQUIRE(spectra, "null spectra");
        if (stages & 1) TFMM_REQUIRE(x, "null x");
        if (stages & 2) TFMM_REQUIRE(y, "null y");
        StreamGuard cs;
        // one eager pass first: first-use allocations and uploads happen outside the capture
        run_stages(plan, stages, x, R, ldx, spectra, apply_weights, beta, y, ldy, cs.s);
        TFMM_CUDA_CHECK(cudaStreamSynchronize(cs.s));
        auto g = std::make_unique<tfmm_graph>();
        g->plan = plan;
        TFMM_CUDA_CHECK(cudaStreamBeginCapture(cs.s, cudaStreamCaptureModeThreadLocal));
        try {
            run_stages(plan, stages, x, R, ldx, spectra, apply_weights, beta, y, ldy, cs.s);
        } catch (...) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(cs.s, &junk);
            if (junk) cudaGraphDestroy(junk);
            throw;
        }
        TFMM_CUDA_CHECK(cudaStreamEndCapture(cs.s, &g->graph));
        TFMM_CUDA_CHECK(cudaGraphInstantiate(&g->exec, g->graph, 0));
        ++plan->p.live_graphs;
        *out = g.release();
    });
}

tfmm_status tfmm_graph_launch(tfmm_graph* graph, void* stream) {
    return guarded([&] {
        TFMM_REQUIRE(graph && graph->exec, "null graph");
        TFMM_CUDA_CHECK(cudaGraphLaunch(graph->exec, (cudaStream_t)stream));
    });
}

tfmm_status tfmm_graph_destroy(tfmm_graph* graph) {
    return guarded([&] {
        if (!graph) return;
        if (graph->exec) cudaGraphExecDestroy(graph->exec);
        if (graph->graph) cudaGraphDestroy(graph->graph);
        if (graph->plan) --graph->plan->p.live_graphs;
        delete graph;
    });
}

tfmm_status tfmm_plan_tuning_get(const tfmm_plan* plan, tfmm_tuning* t) {
    return guarded([&] {
        TFMM_REQUIRE(plan && t, "null argument");
        const Plan& P = plan->p;
        std::memset(t, 0, sizeof(*t));
        t->agg_threads = P.tuning.agg_threads;
        t->agg_ctas_per_sm = P.tuning.agg_ctas_per_sm;
        t->agg_order = P.tuning.agg_order;
        t->dis_threads = P.tuning.dis_threads;
        t->dis_ctas_per_sm = P.tuning.dis_ctas_per_sm;
        t->dis_order = P.tuning.dis_order;
        t->agg_blocks = P.agg_sched.blocks;
        t->dis_blocks = P.dis_sched.blocks;
        t->mrhs_precision = P.params.mrhs_precision;
        t->tc_f34_n1 = P.tc_f34_n1;
        t->tc_dg1a_pairs = P.tc_dg1a_pairs;
        t->single_rhs_split = P.tuning.split;
        t->agg_ms = P.tuned_ms[0];
        t->dis_ms = P.tuned_ms[1];
    });
}

tfmm_status tfmm_plan_tuning_set(tfmm_plan* plan, const tfmm_tuning* t, void* stream) {
    return guarded([&] {
        TFMM_REQUIRE(plan && t, "null argument");
        TFMM_REQUIRE(t->mrhs_precision >= 0 && t->mrhs_precision <= 3, "mrhs_precision must be 0, 1, 2 or 3");
        TFMM_REQUIRE(t->tc_f34_n1 == 0 || (t->tc_f34_n1 >= 16 && t->tc_f34_n1 <= 256 && t->tc_f34_n1 % 16 == 0),
                     "tc_f34_n1 must be 0 or a multiple of 16 in 16..256");
        TFMM_REQUIRE(t->tc_dg1a_pairs == 0 || t->tc_dg1a_pairs == 64 || t->tc_dg1a_pairs == 128,
                     "tc_dg1a_pairs must be 0, 64 or 128");
        TFMM_REQUIRE(t->single_rhs_split >= 0 && t->single_rhs_split <= 2,
                     "single_rhs_split must be 0 (automatic), 1 (always) or 2 (never)");
        if (t->tc_f34_n1 != plan->p.tc_f34_n1 || t->tc_dg1a_pairs != plan->p.tc_dg1a_pairs) {
            TFMM_REQUIRE(plan->p.live_graphs == 0, "destroy the plan's graphs before changing tile shapes");
            plan->p.tc_f34_n1 = t->tc_f34_n1;
            plan->p.tc_dg1a_pairs = t->tc_dg1a_pairs;
            tc_replan_shapes(plan->p);
        }
        HotTuning h;
        h.agg_threads = t->agg_threads; h.agg_ctas_per_sm = t->agg_ctas_per_sm; h.agg_order = t->agg_order;
        h.dis_threads = t->dis_threads; h.dis_ctas_per_sm = t->dis_ctas_per_sm; h.dis_order = t->dis_order;
        h.split = t->single_rhs_split;
        const HotTuning old = plan->p.tuning;
        const bool was_ok = plan->p.hot_ok;
        configure_hot(plan->p, h, (cudaStream_t)stream);
        if (was_ok && !plan->p.hot_ok) {
            configure_hot(plan->p, old, (cudaStream_t)stream);
            fail(TFMM_INVALID_ARG, "launch shape leaves no room for the largest work item");
        }
        plan->p.params.mrhs_precision = t->mrhs_precision;
    });
}

tfmm_status tfmm_autotune(tfmm_plan* plan, int32_t R, double budget_ms, int32_t allow_two_term, void* stream,
                          tfmm_tuning* out) {
    return guarded([&] {
        TFMM_REQUIRE(plan, "null plan");
        Plan& P = plan->p;
        TFMM_REQUIRE(R >= 1 && R <= P.params.max_rhs, "R must be in 1..max_rhs");
        TFMM_REQUIRE(budget_ms > 0, "budget_ms must be positive");
        TFMM_REQUIRE(P.d_factors, "plan has no factors");
        cudaStream_t s = (cudaStream_t)stream;
        const auto t0 = std::chrono::steady_clock::now();
        auto spent = [&] {
            return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        };
        Scratch w;
        const size_t xb = sizeof(float2) * (size_t)P.N * R, sb = sizeof(float2) * (size_t)R * P.G * 2 * P.n_dir;
        TFMM_CUDA_CHECK(device_malloc(&w.x.p, xb));
        TFMM_CUDA_CHECK(device_malloc(&w.spec.p, sb));
        TFMM_CUDA_CHECK(device_malloc(&w.y.p, xb));
        // any finite data times the same: bytes 0x3c give floats of about 0.0115
        TFMM_CUDA_CHECK(cudaMemsetAsync(w.x.p, 0x3c, xb, s));
        TFMM_CUDA_CHECK(cudaMemsetAsync(w.spec.p, 0x3c, sb, s));
        TFMM_CUDA_CHECK(cudaMemsetAsync(w.y.p, 0, xb, s));
        auto* x = static_cast<const tfmm_cfloat*>(w.x.p);
        auto* sp = static_cast<tfmm_cfloat*>(w.spec.p);
        auto* y = static_cast<tfmm_cfloat*>(w.y.p);
        const tfmm_cfloat zero{0.f, 0.f};
        Timer tm;
        auto agg = [&] { run_stages(plan, 1, x, R, P.N, sp, 1, zero, y, P.N, s); };
        auto dis = [&] { run_stages(plan, 2, x, R, P.N, sp, 1, zero, y, P.N, s); };
        if (R == 1 && P.hot_ok) {
            // launch shape x queue order, one stage at a time; the other stage keeps its setting
            HotTuning best = P.tuning;
            double best_ms[2] = {1e30, 1e30};
            const int threads[3] = {512, 384, 256};
            const int ctas[3] = {0, 2, 1};
            for (int stage = 0; stage < 2; ++stage) {
                std::vector<std::pair<int, int>> seen;  // (threads and order, blocks) already timed
                for (int order = 0; order < 2; ++order)
                    for (int nt : threads)
                        for (int c : ctas) {
                            // the budget stops the search once this stage has one timing
                            if (spent() > budget_ms * (stage + 1) / 2 && best_ms[stage] < 1e30) continue;
                            HotTuning t = best;
                            (stage == 0 ? t.agg_threads : t.dis_threads) = nt;
                            (stage == 0 ? t.agg_ctas_per_sm : t.dis_ctas_per_sm) = c;
                            (stage == 0 ? t.agg_order : t.dis_order) = order;
                            configure_hot(P, t, s);
                            if (!P.hot_ok) continue;
                            const Schedule& sc = stage == 0 ? P.agg_sched : P.dis_sched;
                            if (std::find(seen.begin(), seen.end(), std::make_pair(nt * 2 + order, sc.blocks)) !=
                                seen.end())
                                continue;
                            seen.emplace_back(nt * 2 + order, sc.blocks);
                            const double ms = stage == 0 ? time_ms(agg, 5, s, tm) : time_ms(dis, 5, s, tm);
                            if (ms < best_ms[stage]) {
                                best_ms[stage] = ms;
                                best = t;
                            }
                        }
            }
            configure_hot(P, best, s);
            P.tuned_ms[0] = best_ms[0];
            P.tuned_ms[1] = best_ms[1];
        } else if (R > 1) {
            // the multi-RHS engine: 3-term split-BF16 chain, FP32 CUDA-core chain, the single-RHS
            // kernels column by column, and on request the 2-term split
            std::vector<int> cand = {3, 0};
            if (P.hot_ok) cand.push_back(1);
            if (allow_two_term) cand.push_back(2);
            int best = P.params.mrhs_precision;
            double best_ms = 1e30, ba = 0, bd = 0;
            for (int prec : cand) {
                if (spent() > budget_ms && best_ms < 1e30) break;
                P.params.mrhs_precision = prec;
                const double a = time_ms(agg, 2, s, tm);
                const double d = time_ms(dis, 2, s, tm);
                if (a + d < best_ms) {
                    best_ms = a + d;
                    best = prec;
                    ba = a;
                    bd = d;
                }
            }
            P.params.mrhs_precision = best;
            P.tuned_ms[0] = ba;
            P.tuned_ms[1] = bd;
            if ((best == 2 || best == 3) && P.live_graphs == 0) {
                // tile shapes of the tensor-core chain: fused AG3+AG4 block size x DG1a pairs
                int bn1 = P.tc_f34_n1, bpairs = P.tc_dg1a_pairs;
                for (int n1 : {0, 128, 64})
                    for (int pairs : {0, 64}) {
                        if (spent() > budget_ms) break;
                        if (n1 == bn1 && pairs == bpairs) continue;
                        P.tc_f34_n1 = n1;
                        P.tc_dg1a_pairs = pairs;
                        tc_replan_shapes(P);
                        const double a = time_ms(agg, 2, s, tm);
                        const double d = time_ms(dis, 2, s, tm);
                        if (a + d < best_ms) {
                            best_ms = a + d;
                            bn1 = n1;
                            bpairs = pairs;
                            P.tuned_ms[0] = a;
                            P.tuned_ms[1] = d;
                        }
                    }
                if (P.tc_f34_n1 != bn1 || P.tc_dg1a_pairs != bpairs) {
                    P.tc_f34_n1 = bn1;
                    P.tc_dg1a_pairs = bpairs;
                    tc_replan_shapes(P);
                }
            }
        }
        TFMM_CUDA_CHECK(cudaStreamSynchronize(s));
        if (out && tfmm_plan_tuning_get(plan, out) != TFMM_OK) fail(TFMM_INVALID_ARG, last_error());
    });
}

}  // extern "C"
