// C ABI of the tfmm library: argument checking, mesh / RWG construction,
// box grouping, spherical grid, plan bookkeeping.  Every entry point catches
// internal errors and returns a status code.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <numeric>
#include <string>
#include <tuple>

#include <atomic>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"

namespace tfmm {

std::string& last_error() {
    thread_local std::string msg;
    return msg;
}

void upload_common(Plan& P, cudaStream_t s) {
    int dev = 0;
    TFMM_CUDA_CHECK(cudaGetDevice(&dev));
    TFMM_CUDA_CHECK(cudaDeviceGetAttribute(&P.num_sms, cudaDevAttrMultiProcessorCount, dev));
    std::vector<int> ids(P.grp_rwg.begin(), P.grp_rwg.end());
    TFMM_CUDA_CHECK(device_malloc(&P.d_grp_rwg, sizeof(int) * std::max<int64_t>(P.N, 1)));
    TFMM_CUDA_CHECK(cudaMemcpyAsync(P.d_grp_rwg, ids.data(), sizeof(int) * P.N, cudaMemcpyHostToDevice, s));
    TFMM_CUDA_CHECK(device_malloc(&P.d_weights, sizeof(float) * P.n_dir));
    TFMM_CUDA_CHECK(cudaMemcpyAsync(P.d_weights, P.weights.data(), sizeof(float) * P.n_dir, cudaMemcpyHostToDevice, s));
    TFMM_CUDA_CHECK(device_malloc(&P.d_counters, sizeof(unsigned) * 16));
    TFMM_CUDA_CHECK(cudaMemsetAsync(P.d_counters, 0, sizeof(unsigned) * 16, s));
    TFMM_CUDA_CHECK(cudaStreamSynchronize(s));
}

namespace {

// RWG functions (Sec. II.A, ref. [20]): every edge shared by exactly two
// triangles; RWGs sorted by (min, max) vertex id; T+ the lower triangle id.
void build_rwg(Mesh& M) {
    struct HalfEdge {
        int64_t a, b, t, f;
    };
    std::vector<HalfEdge> he;
    he.reserve((size_t)M.nt * 3);
    for (int64_t t = 0; t < M.nt; ++t) {
        const int32_t* v = &M.tris[3 * t];
        for (int e = 0; e < 3; ++e) {
            const int64_t u = v[e], w = v[(e + 1) % 3], f = v[(e + 2) % 3];
            he.push_back({std::min(u, w), std::max(u, w), t, f});
        }
    }
    std::sort(he.begin(), he.end(), [](const HalfEdge& x, const HalfEdge& y) {
        return std::tie(x.a, x.b, x.t) < std::tie(y.a, y.b, y.t);
    });
    M.edge.clear(); M.tri.clear(); M.freev.clear(); M.length.clear();
    size_t i = 0;
    while (i < he.size()) {
        size_t j = i;
        while (j < he.size() && he[j].a == he[i].a && he[j].b == he[i].b) ++j;
        if (j - i == 2) {
            M.edge.push_back(he[i].a); M.edge.push_back(he[i].b);
            M.tri.push_back(he[i].t); M.tri.push_back(he[i + 1].t);
            M.freev.push_back(he[i].f); M.freev.push_back(he[i + 1].f);
            const double* pa = &M.verts[3 * he[i].a];
            const double* pb = &M.verts[3 * he[i].b];
            const double dx = pb[0] - pa[0], dy = pb[1] - pa[1], dz = pb[2] - pa[2];
            M.length.push_back(std::sqrt(dx * dx + dy * dy + dz * dz));
        }
        i = j;
    }
    M.n_rwg = (int64_t)M.length.size();
}

// L = kd + 1.8 d0^(2/3) (kd)^(1/3), d = a sqrt(3), rounded up (Sec. II.A, ref. [25]).
int bandwidth(double k, double box, double digits) {
    const double kd = k * box * std::sqrt(3.0);
    return (int)std::ceil(kd + 1.8 * std::pow(digits, 2.0 / 3.0) * std::pow(kd, 1.0 / 3.0));
}

void setup_grid(Plan& P, int L, int nphi_rule) {
    P.L = L;
    P.n_theta = L + 1;
    P.n_phi = nphi_rule == 0 ? 2 * L + 1 : 2 * L + 2;
    P.n_dir = P.n_theta * P.n_phi;
    P.ld_dir = (int)round_up(P.n_dir, 2);
    std::vector<double> x, w;
    gauss_legendre(P.n_theta, x, w);
    // theta ascending <=> cos(theta) descending
    P.theta.resize(P.n_theta);
    P.w_theta.resize(P.n_theta);
    for (int i = 0; i < P.n_theta; ++i) {
        P.theta[i] = std::acos(x[P.n_theta - 1 - i]);
        P.w_theta[i] = w[P.n_theta - 1 - i];
    }
    const double pi = 3.14159265358979323846;
    P.phi.resize(P.n_phi);
    for (int j = 0; j < P.n_phi; ++j) P.phi[j] = 2.0 * pi * j / P.n_phi;
    P.w_phi = 2.0 * pi / P.n_phi;
    P.weights.resize(P.n_dir);
    for (int ip = 0; ip < P.n_phi; ++ip)
        for (int it = 0; it < P.n_theta; ++it) P.weights[it + P.n_theta * ip] = (float)(P.w_theta[it] * P.w_phi);
}

// Box grid of edge a anchored at the minimum corner of the RWG midpoints;
// groups are the non-empty boxes in ascending ix + Kx (iy + Ky iz).
void make_groups(Plan& P, const Mesh& M, double box) {
    const int64_t N = M.n_rwg;
    std::vector<double> mp((size_t)N * 3);
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t n = 0; n < N; ++n)
        for (int c = 0; c < 3; ++c) {
            const double v = 0.5 * (M.verts[3 * M.edge[2 * n] + c] + M.verts[3 * M.edge[2 * n + 1] + c]);
            mp[3 * n + c] = v;
            lo[c] = std::min(lo[c], v);
            hi[c] = std::max(hi[c], v);
        }
    for (int c = 0; c < 3; ++c) P.K[c] = std::max(1, (int)std::ceil((hi[c] - lo[c]) / box));
    std::vector<int64_t> lin(N);
    for (int64_t n = 0; n < N; ++n) {
        int64_t idx[3];
        for (int c = 0; c < 3; ++c) {
            int64_t v = (int64_t)std::floor((mp[3 * n + c] - lo[c]) / box);
            idx[c] = std::min<int64_t>(std::max<int64_t>(v, 0), P.K[c] - 1);
        }
        lin[n] = idx[0] + (int64_t)P.K[0] * (idx[1] + (int64_t)P.K[1] * idx[2]);
    }
    std::vector<int64_t> order(N);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return lin[a] < lin[b]; });
    P.grp_off.clear();
    P.grp_rwg = order;
    P.centres.clear();
    for (int64_t i = 0; i < N; ++i) {
        if (i == 0 || lin[order[i]] != lin[order[i - 1]]) {
            P.grp_off.push_back(i);
            const int64_t b = lin[order[i]];
            const int64_t bi[3] = {b % P.K[0], (b / P.K[0]) % P.K[1], b / ((int64_t)P.K[0] * P.K[1])};
            for (int c = 0; c < 3; ++c) P.centres.push_back(lo[c] + (bi[c] + 0.5) * box);
        }
    }
    P.grp_off.push_back(N);
    P.G = (int)P.grp_off.size() - 1;
    P.N = N;
}


void check_params(const tfmm_params& p) {
    TFMM_REQUIRE(std::isfinite(p.k) && p.k > 0, "k must be positive");
    TFMM_REQUIRE(std::isfinite(p.box) && p.box > 0, "box must be positive");
    TFMM_REQUIRE(std::isfinite(p.digits) && p.digits > 0, "digits must be positive");
    TFMM_REQUIRE(p.nphi_rule == 0 || p.nphi_rule == 1, "nphi_rule must be 0 (2L+1) or 1 (2L+2)");
    TFMM_REQUIRE(p.L_override >= 0 && p.L_override <= 1000, "L_override out of range");
    TFMM_REQUIRE(std::isfinite(p.tol) && p.tol >= 0, "tol must be >= 0");
    TFMM_REQUIRE(p.quad_order >= 1 && p.quad_order <= 10, "quad_order must be in 1..10");
    TFMM_REQUIRE(p.max_rhs >= 1, "max_rhs must be >= 1");
    TFMM_REQUIRE(p.batch_groups >= 0, "batch_groups must be >= 0");
    TFMM_REQUIRE(p.mrhs_precision >= 0 && p.mrhs_precision <= 3, "mrhs_precision must be 0, 1, 2 or 3");
    TFMM_REQUIRE(p.compression == 0 || p.compression == 1, "compression must be 0 (Tucker) or 1 (SVD)");
}

// The engine that applies one call with R columns:
//   columns: the persistent single-RHS kernels, one column after the other (R = 1, or
//            mrhs_precision 1, or TFMM_MR=loop);
//   chain:   the grouped-GEMM chain on FP32 CUDA cores (mrhs_precision 0), also the
//            fallback when a work item does not fit the single-RHS kernels;
//   tc:      the split-BF16 tensor-core chain with `terms` terms (mrhs_precision 2, 3).
enum class Engine { columns, chain, tc };

Engine engine_for(const Plan& P, int R, int* terms) {
    *terms = 0;
    const int p = P.params.mrhs_precision;
    const char* e = std::getenv("TFMM_MR");
    const bool loop = e && std::strcmp(e, "loop") == 0;
    if (P.hot_ok && (R <= 1 || loop || p == 1 || plan_is_svd(P))) return Engine::columns;
    if (R > 1 && (p == 2 || p == 3)) {
        *terms = p;
        return Engine::tc;
    }
    return Engine::chain;
}

// An NVTX range around one hot-path call (seen by profilers, free otherwise).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

void run_aggregate(Plan& P, const float2* x, int R, int64_t ldx, float2* spec, cudaStream_t s) {
    NvtxRange nvtx("tfmm_aggregate");
    int T = 0;
    switch (engine_for(P, R, &T)) {
        case Engine::tc: launch_tc_aggregate(P, T, x, R, ldx, spec, s); break;
        case Engine::chain: launch_mr_aggregate(P, x, R, ldx, spec, s); break;
        default: launch_tucker_aggregate(P, x, R, ldx, spec, s);
    }
}

void run_disaggregate(Plan& P, const float2* spec, int R, int weights, float2 beta, float2* y, int64_t ldy,
                      cudaStream_t s) {
    NvtxRange nvtx("tfmm_disaggregate");
    int T = 0;
    switch (engine_for(P, R, &T)) {
        case Engine::tc: launch_tc_disaggregate(P, T, spec, R, weights, beta, y, ldy, s); break;
        case Engine::chain: launch_mr_disaggregate(P, spec, R, weights, beta, y, ldy, s); break;
        default: launch_tucker_disaggregate(P, spec, R, weights, beta, y, ldy, s);
    }
}

void check_hot(const Plan& P, const void* a, const void* b, int R, int64_t ld) {
    TFMM_REQUIRE(a != nullptr && b != nullptr, "null buffer");
    TFMM_REQUIRE(R >= 1 && R <= P.params.max_rhs, "R must be in 1..max_rhs");
    TFMM_REQUIRE(ld >= P.N, "leading dimension smaller than n_rwg");
    TFMM_REQUIRE(P.d_factors != nullptr, "plan has no factors");
}

}  // namespace
}  // namespace tfmm

namespace tfmm {

namespace {
// Allocations left before the one the test hook fails (0: disarmed).
std::atomic<int64_t> g_fail_alloc_in{0};
}  // namespace

cudaError_t device_malloc_bytes(void** p, size_t bytes) {
    if (g_fail_alloc_in.load() > 0 && g_fail_alloc_in.fetch_sub(1) == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

}  // namespace tfmm

using namespace tfmm;

extern "C" {

tfmm_status tfmm_test_fail_allocation(int64_t nth) {
    return guarded([&] {
        TFMM_REQUIRE(nth >= 0, "nth must be >= 0");
        g_fail_alloc_in.store(nth);
    });
}

const char* tfmm_last_error(void) { return last_error().c_str(); }

tfmm_status tfmm_params_default(tfmm_params* p) {
    return guarded([&] {
        TFMM_REQUIRE(p, "null params");
        std::memset(p, 0, sizeof(*p));
        p->k = 2.0 * 3.14159265358979323846;
        p->box = 0.5;
        p->digits = 3.0;
        p->nphi_rule = 1;
        p->L_override = 0;
        p->tol = 1e-4;
        p->quad_order = 5;
        p->keep_dense = 0;
        p->max_rhs = 1;
        p->batch_groups = 0;
    });
}

tfmm_status tfmm_mesh_create(const double* verts, int64_t nv, const int32_t* tris, int64_t nt, tfmm_mesh** out) {
    return guarded([&] {
        TFMM_REQUIRE(out, "null output");
        *out = nullptr;
        TFMM_REQUIRE(verts && tris, "null mesh arrays");
        TFMM_REQUIRE(nv >= 3 && nt >= 1, "mesh needs at least 3 vertices and 1 triangle");
        TFMM_REQUIRE(nv < (int64_t)1 << 31 && nt < (int64_t)1 << 31, "mesh too large");
        auto h = std::make_unique<tfmm_mesh>();
        Mesh& M = h->m;
        M.nv = nv;
        M.nt = nt;
        M.verts.assign(verts, verts + 3 * nv);
        M.tris.assign(tris, tris + 3 * nt);
        for (int64_t i = 0; i < 3 * nv; ++i) TFMM_REQUIRE(std::isfinite(M.verts[i]), "non-finite vertex coordinate");
        for (int64_t t = 0; t < nt; ++t) {
            const int32_t a = M.tris[3 * t], b = M.tris[3 * t + 1], c = M.tris[3 * t + 2];
            TFMM_REQUIRE(a >= 0 && a < nv && b >= 0 && b < nv && c >= 0 && c < nv,
                         "triangle " + std::to_string(t) + " has an out-of-range vertex id");
            TFMM_REQUIRE(a != b && b != c && a != c, "triangle " + std::to_string(t) + " repeats a vertex");
            const double* pa = &M.verts[3 * a];
            const double* pb = &M.verts[3 * b];
            const double* pc = &M.verts[3 * c];
            const double u[3] = {pb[0] - pa[0], pb[1] - pa[1], pb[2] - pa[2]};
            const double v[3] = {pc[0] - pa[0], pc[1] - pa[1], pc[2] - pa[2]};
            const double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
            TFMM_REQUIRE(cx * cx + cy * cy + cz * cz > 0, "triangle " + std::to_string(t) + " is degenerate");
        }
        build_rwg(M);
        *out = h.release();
    });
}

tfmm_status tfmm_mesh_num_rwg(const tfmm_mesh* mesh, int64_t* n_rwg) {
    return guarded([&] {
        TFMM_REQUIRE(mesh && n_rwg, "null argument");
        *n_rwg = mesh->m.n_rwg;
    });
}

tfmm_status tfmm_mesh_rwg(const tfmm_mesh* mesh, int64_t* edge, int64_t* tri, int64_t* free_vertex) {
    return guarded([&] {
        TFMM_REQUIRE(mesh, "null mesh");
        const Mesh& M = mesh->m;
        if (edge) std::copy(M.edge.begin(), M.edge.end(), edge);
        if (tri) std::copy(M.tri.begin(), M.tri.end(), tri);
        if (free_vertex) std::copy(M.freev.begin(), M.freev.end(), free_vertex);
    });
}

tfmm_status tfmm_mesh_destroy(tfmm_mesh* mesh) {
    return guarded([&] { delete mesh; });
}

tfmm_status tfmm_plan_create(const tfmm_mesh* mesh, const tfmm_params* prm, void* stream, tfmm_plan** out) {
    return guarded([&] {
        TFMM_REQUIRE(out, "null output");
        *out = nullptr;
        TFMM_REQUIRE(mesh && prm, "null argument");
        check_params(*prm);
        const Mesh& M = mesh->m;
        TFMM_REQUIRE(M.n_rwg >= 1, "mesh has no RWG functions (no interior edges)");
        cudaStream_t s = (cudaStream_t)stream;
        auto h = std::make_unique<tfmm_plan>();
        Plan& P = h->p;
        P.params = *prm;
        P.k = prm->k;
        const int L = prm->L_override > 0 ? prm->L_override : bandwidth(prm->k, prm->box, prm->digits);
        setup_grid(P, L, prm->nphi_rule);
        make_groups(P, M, prm->box);
        P.has_geometry = true;
        P.geom.resize(P.N);
        for (int64_t n = 0; n < P.N; ++n) {
            RwgGeom& g = P.geom[n];
            for (int c = 0; c < 3; ++c) {
                g.pp[c] = M.verts[3 * M.freev[2 * n] + c];
                g.pm[c] = M.verts[3 * M.freev[2 * n + 1] + c];
                g.q1[c] = M.verts[3 * M.edge[2 * n] + c];
                g.q2[c] = M.verts[3 * M.edge[2 * n + 1] + c];
            }
            g.l = M.length[n];
            g.pad[0] = g.pad[1] = g.pad[2] = 0.0;
        }
        upload_common(P, s);
        build_tucker_setup(P, M, s);
        if (prm->keep_dense) finalize_dense_layout(P);
        *out = h.release();
    });
}

tfmm_status tfmm_plan_from_tucker(int64_t n_rwg, int32_t n_groups, int32_t n_theta, int32_t n_phi,
                                  const int64_t* group_offsets, const int64_t* group_rwg, const int32_t* ranks,
                                  const tfmm_cdouble* factors, const double* weights, int32_t max_rhs, void* stream,
                                  tfmm_plan** out) {
    return guarded([&] {
        TFMM_REQUIRE(out, "null output");
        *out = nullptr;
        TFMM_REQUIRE(group_offsets && group_rwg && ranks && factors, "null argument");
        TFMM_REQUIRE(n_rwg >= 1 && n_rwg < ((int64_t)1 << 31), "n_rwg out of range");
        TFMM_REQUIRE(n_groups >= 1 && n_theta >= 1 && n_phi >= 1, "sizes must be positive");
        TFMM_REQUIRE(max_rhs >= 1, "max_rhs must be >= 1");
        cudaStream_t s = (cudaStream_t)stream;
        auto h = std::make_unique<tfmm_plan>();
        Plan& P = h->p;
        tfmm_params_default(&P.params);
        P.params.max_rhs = max_rhs;
        P.n_theta = n_theta;
        P.n_phi = n_phi;
        P.L = n_theta - 1;
        P.n_dir = n_theta * n_phi;
        P.ld_dir = (int)round_up(P.n_dir, 2);
        P.G = n_groups;
        P.N = n_rwg;
        P.grp_off.assign(group_offsets, group_offsets + n_groups + 1);
        TFMM_REQUIRE(P.grp_off[0] == 0, "group_offsets[0] must be 0");
        for (int g = 0; g < n_groups; ++g) TFMM_REQUIRE(P.grp_off[g + 1] > P.grp_off[g], "empty or unordered group");
        const int64_t total = P.grp_off[n_groups];
        TFMM_REQUIRE(total == n_rwg, "every RWG must belong to exactly one group");
        P.grp_rwg.assign(group_rwg, group_rwg + total);
        std::vector<char> seen(n_rwg, 0);
        for (int64_t v : P.grp_rwg) {
            TFMM_REQUIRE(v >= 0 && v < n_rwg, "group member out of range");
            TFMM_REQUIRE(!seen[v], "RWG listed in two groups");
            seen[v] = 1;
        }
        P.ranks.assign(ranks, ranks + (size_t)n_groups * 6);
        P.weights.assign(P.n_dir, 1.0f);
        if (weights)
            for (int i = 0; i < P.n_dir; ++i) P.weights[i] = (float)weights[i];
        upload_common(P, s);
        P.f64.assign((size_t)n_groups * 2, HostFactors64{});
        const double2* src = reinterpret_cast<const double2*>(factors);
        int64_t pos = 0;
        for (int g = 0; g < n_groups; ++g) {
            const int64_t nb = P.grp_off[g + 1] - P.grp_off[g];
            for (int al = 0; al < 2; ++al) {
                const int* rk = &P.ranks[((size_t)g * 2 + al) * 3];
                TFMM_REQUIRE(rk[0] >= 1 && rk[0] <= n_theta && rk[1] >= 1 && rk[1] <= n_phi && rk[2] >= 1 && rk[2] <= nb,
                             "rank out of range for group " + std::to_string(g));
                pos += (int64_t)n_theta * rk[0] + (int64_t)n_phi * rk[1] + nb * rk[2] + (int64_t)rk[0] * rk[1] * rk[2];
            }
        }
        double2* arena = nullptr;
        TFMM_CUDA_CHECK(device_malloc(&arena, sizeof(double2) * pos));
        P.f64_arenas.push_back(arena);
        TFMM_CUDA_CHECK(cudaMemcpyAsync(arena, src, sizeof(double2) * pos, cudaMemcpyHostToDevice, s));
        pos = 0;
        for (int g = 0; g < n_groups; ++g) {
            const int64_t nb = P.grp_off[g + 1] - P.grp_off[g];
            for (int al = 0; al < 2; ++al) {
                const int* rk = &P.ranks[((size_t)g * 2 + al) * 3];
                HostFactors64& F = P.f64[(size_t)g * 2 + al];
                F.rt = rk[0]; F.rp = rk[1]; F.rb = rk[2];
                F.base = arena + pos;
                pos += (int64_t)n_theta * rk[0] + (int64_t)n_phi * rk[1] + nb * rk[2] + (int64_t)rk[0] * rk[1] * rk[2];
            }
        }
        pack_factors_fp32(P, s);
        TFMM_CUDA_CHECK(cudaStreamSynchronize(s));
        *out = h.release();
    });
}

tfmm_status tfmm_plan_set_dense(tfmm_plan* plan, const tfmm_cdouble* tensors, void* stream) {
    return guarded([&] {
        TFMM_REQUIRE(plan && tensors, "null argument");
        Plan& P = plan->p;
        cudaStream_t s = (cudaStream_t)stream;
        if (!P.d_dense) {
            P.dense_elems = (int64_t)P.ld_dir * P.N * 2;
            TFMM_CUDA_CHECK(device_malloc(&P.d_dense, sizeof(float2) * P.dense_elems));
        }
        TFMM_CUDA_CHECK(cudaMemsetAsync(P.d_dense, 0, sizeof(float2) * P.dense_elems, s));
        const double2* src = reinterpret_cast<const double2*>(tensors);
        int64_t pos = 0;
        double2* tmp = nullptr;
        int64_t max_e = 0;
        for (int g = 0; g < P.G; ++g) max_e = std::max<int64_t>(max_e, (P.grp_off[g + 1] - P.grp_off[g]) * P.n_dir);
        TFMM_CUDA_CHECK(device_malloc(&tmp, sizeof(double2) * max_e));
        struct Free { double2* p; ~Free() { cudaFree(p); } } fr{tmp};
        for (int g = 0; g < P.G; ++g)
            for (int al = 0; al < 2; ++al) {
                const int64_t e = (P.grp_off[g + 1] - P.grp_off[g]) * P.n_dir;
                TFMM_CUDA_CHECK(cudaMemcpyAsync(tmp, src + pos, sizeof(double2) * e, cudaMemcpyHostToDevice, s));
                pack_dense_fp32_from_f64(P, tmp, g, al, s);
                TFMM_CUDA_CHECK(cudaStreamSynchronize(s));
                pos += e;
            }
        if (!P.d_dense_items) finalize_dense_layout(P);
    });
}

tfmm_status tfmm_plan_info_get(const tfmm_plan* plan, tfmm_plan_info* info) {
    return guarded([&] {
        TFMM_REQUIRE(plan && info, "null argument");
        const Plan& P = plan->p;
        std::memset(info, 0, sizeof(*info));
        info->L = P.L;
        info->n_theta = P.n_theta;
        info->n_phi = P.n_phi;
        info->n_dir = P.n_dir;
        info->n_groups = P.G;
        for (int c = 0; c < 3; ++c) info->K[c] = P.K[c];
        info->n_rwg = P.N;
        info->max_n_beta = P.max_nb;
        for (int c = 0; c < 3; ++c) info->max_rank[c] = P.max_rank[c];
        info->tucker_bytes = P.factor_elems * (int64_t)sizeof(float2);
        info->tucker_bytes_alg = P.factor_elems_alg * (int64_t)sizeof(float2);
        info->dense_bytes = P.d_dense ? P.dense_elems * (int64_t)sizeof(float2) : 0;
        for (int c = 0; c < 4; ++c) info->setup_ms[c] = P.setup_ms[c];
        if (P.tc_err.p) TFMM_CUDA_CHECK(cudaMemcpy(&info->kernel_errors, P.tc_err.p, sizeof(int), cudaMemcpyDeviceToHost));
    });
}

tfmm_status tfmm_plan_set_mrhs_precision(tfmm_plan* plan, int32_t precision) {
    return guarded([&] {
        TFMM_REQUIRE(plan, "null plan");
        TFMM_REQUIRE(precision >= 0 && precision <= 3, "mrhs_precision must be 0, 1, 2 or 3");
        plan->p.params.mrhs_precision = precision;
    });
}

tfmm_status tfmm_plan_group(const tfmm_plan* plan, int32_t g, int32_t alpha, int64_t* n_beta, int32_t* ranks3) {
    return guarded([&] {
        TFMM_REQUIRE(plan, "null plan");
        const Plan& P = plan->p;
        TFMM_REQUIRE(g >= 0 && g < P.G && (alpha == 0 || alpha == 1), "group or alpha out of range");
        if (n_beta) *n_beta = P.grp_off[g + 1] - P.grp_off[g];
        if (ranks3)
            for (int c = 0; c < 3; ++c) ranks3[c] = P.ranks[((size_t)g * 2 + alpha) * 3 + c];
    });
}

tfmm_status tfmm_plan_members(const tfmm_plan* plan, int64_t* offsets, int64_t* rwg_ids) {
    return guarded([&] {
        TFMM_REQUIRE(plan, "null plan");
        const Plan& P = plan->p;
        if (offsets) std::copy(P.grp_off.begin(), P.grp_off.end(), offsets);
        if (rwg_ids) std::copy(P.grp_rwg.begin(), P.grp_rwg.end(), rwg_ids);
    });
}

tfmm_status tfmm_plan_centres(const tfmm_plan* plan, double* centres) {
    return guarded([&] {
        TFMM_REQUIRE(plan && centres, "null argument");
        TFMM_REQUIRE(plan->p.has_geometry, "plan was built from factors and has no box centres");
        std::copy(plan->p.centres.begin(), plan->p.centres.end(), centres);
    });
}

tfmm_status tfmm_plan_quadrature(const tfmm_plan* plan, double* theta, double* w_theta, double* phi, double* w_phi) {
    return guarded([&] {
        TFMM_REQUIRE(plan, "null plan");
        const Plan& P = plan->p;
        TFMM_REQUIRE(!P.theta.empty(), "plan was built from factors and has no grid");
        if (theta) std::copy(P.theta.begin(), P.theta.end(), theta);
        if (w_theta) std::copy(P.w_theta.begin(), P.w_theta.end(), w_theta);
        if (phi) std::copy(P.phi.begin(), P.phi.end(), phi);
        if (w_phi) *w_phi = P.w_phi;
    });
}

tfmm_status tfmm_plan_export_factors(const tfmm_plan* plan, int32_t g, int32_t alpha, tfmm_cdouble* U_theta,
                                     tfmm_cdouble* U_phi, tfmm_cdouble* U_beta, tfmm_cdouble* core) {
    return guarded([&] {
        TFMM_REQUIRE(plan, "null plan");
        const Plan& P = plan->p;
        TFMM_REQUIRE(g >= 0 && g < P.G && (alpha == 0 || alpha == 1), "group or alpha out of range");
        const HostFactors64& F = P.f64[(size_t)g * 2 + alpha];
        const int64_t nb = P.grp_off[g + 1] - P.grp_off[g];
        const int64_t e_ut = (int64_t)P.n_theta * F.rt, e_up = (int64_t)P.n_phi * F.rp, e_ub = nb * F.rb,
                      e_c = (int64_t)F.rt * F.rp * F.rb;
        const double2* b = F.base;
        if (U_theta) TFMM_CUDA_CHECK(cudaMemcpy(U_theta, b, 16 * e_ut, cudaMemcpyDeviceToHost));
        if (U_phi) TFMM_CUDA_CHECK(cudaMemcpy(U_phi, b + e_ut, 16 * e_up, cudaMemcpyDeviceToHost));
        if (U_beta) TFMM_CUDA_CHECK(cudaMemcpy(U_beta, b + e_ut + e_up, 16 * e_ub, cudaMemcpyDeviceToHost));
        if (core) TFMM_CUDA_CHECK(cudaMemcpy(core, b + e_ut + e_up + e_ub, 16 * e_c, cudaMemcpyDeviceToHost));
    });
}

tfmm_status tfmm_plan_farfield(const tfmm_plan* plan, int32_t g, tfmm_cdouble* A_theta, tfmm_cdouble* A_phi,
                               void* stream) {
    return guarded([&] {
        TFMM_REQUIRE(plan && A_theta && A_phi, "null argument");
        farfield_group_host(plan->p, g, reinterpret_cast<double2*>(A_theta), reinterpret_cast<double2*>(A_phi),
                            (cudaStream_t)stream);
    });
}

tfmm_status tfmm_plan_destroy(tfmm_plan* plan) {
    return guarded([&] {
        if (plan) TFMM_REQUIRE(plan->p.live_graphs == 0, "destroy the plan's graphs first");
        delete plan;
    });
}

tfmm_status tfmm_aggregate(tfmm_plan* plan, const tfmm_cfloat* x, int32_t R, int64_t ldx, tfmm_cfloat* spectra,
                           void* stream) {
    return guarded([&] {
        TFMM_REQUIRE(plan, "null plan");
        check_hot(plan->p, x, spectra, R, ldx);
        run_aggregate(plan->p, reinterpret_cast<const float2*>(x), R, ldx, reinterpret_cast<float2*>(spectra),
                      (cudaStream_t)stream);
    });
}

tfmm_status tfmm_disaggregate(tfmm_plan* plan, const tfmm_cfloat* spectra, int32_t R, int32_t apply_weights,
                              tfmm_cfloat beta, tfmm_cfloat* y, int64_t ldy, void* stream) {
    return guarded([&] {
        TFMM_REQUIRE(plan, "null plan");
        check_hot(plan->p, spectra, y, R, ldy);
        run_disaggregate(plan->p, reinterpret_cast<const float2*>(spectra), R, apply_weights,
                         make_float2(beta.re, beta.im), reinterpret_cast<float2*>(y), ldy, (cudaStream_t)stream);
    });
}

tfmm_status tfmm_aggregate_dense(tfmm_plan* plan, const tfmm_cfloat* x, int32_t R, int64_t ldx, tfmm_cfloat* spectra,
                                 void* stream) {
    return guarded([&] {
        TFMM_REQUIRE(plan, "null plan");
        check_hot(plan->p, x, spectra, R, ldx);
        if (!plan->p.d_dense || !plan->p.d_dense_items) fail(TFMM_NOT_BUILT, "plan holds no dense tensors");
        launch_dense_aggregate(plan->p, reinterpret_cast<const float2*>(x), R, ldx, reinterpret_cast<float2*>(spectra),
                               (cudaStream_t)stream);
    });
}

tfmm_status tfmm_disaggregate_dense(tfmm_plan* plan, const tfmm_cfloat* spectra, int32_t R, int32_t apply_weights,
                                    tfmm_cfloat beta, tfmm_cfloat* y, int64_t ldy, void* stream) {
    return guarded([&] {
        TFMM_REQUIRE(plan, "null plan");
        check_hot(plan->p, spectra, y, R, ldy);
        if (!plan->p.d_dense || !plan->p.d_dense_items) fail(TFMM_NOT_BUILT, "plan holds no dense tensors");
        launch_dense_disaggregate(plan->p, reinterpret_cast<const float2*>(spectra), R, apply_weights,
                                  make_float2(beta.re, beta.im), reinterpret_cast<float2*>(y), ldy,
                                  (cudaStream_t)stream);
    });
}

tfmm_status tfmm_matvec_host(tfmm_plan* plan, const tfmm_cfloat* x_host, tfmm_cfloat* y_host, int32_t R, int32_t dense,
                             void* stream) {
    return guarded([&] {
        TFMM_REQUIRE(plan && x_host && y_host, "null argument");
        Plan& P = plan->p;
        TFMM_REQUIRE(R >= 1 && R <= P.params.max_rhs, "R must be in 1..max_rhs");
        if (dense && (!P.d_dense || !P.d_dense_items)) fail(TFMM_NOT_BUILT, "plan holds no dense tensors");
        cudaStream_t s = (cudaStream_t)stream;
        if (P.ws_R < R) {
            cudaFree(P.d_ws_x); cudaFree(P.d_ws_spec); cudaFree(P.d_ws_y);
            P.d_ws_x = P.d_ws_spec = P.d_ws_y = nullptr;
            P.ws_R = 0;
            TFMM_CUDA_CHECK(device_malloc(&P.d_ws_x, sizeof(float2) * P.N * R));
            TFMM_CUDA_CHECK(device_malloc(&P.d_ws_y, sizeof(float2) * P.N * R));
            TFMM_CUDA_CHECK(device_malloc(&P.d_ws_spec, sizeof(float2) * (int64_t)R * P.G * 2 * P.n_dir));
            P.ws_R = R;
        }
        TFMM_CUDA_CHECK(cudaMemcpyAsync(P.d_ws_x, x_host, sizeof(float2) * P.N * R, cudaMemcpyHostToDevice, s));
        const float2 zero = make_float2(0.f, 0.f);
        if (dense) {
            launch_dense_aggregate(P, P.d_ws_x, R, P.N, P.d_ws_spec, s);
            launch_dense_disaggregate(P, P.d_ws_spec, R, 1, zero, P.d_ws_y, P.N, s);
        } else {
            run_aggregate(P, P.d_ws_x, R, P.N, P.d_ws_spec, s);
            run_disaggregate(P, P.d_ws_spec, R, 1, zero, P.d_ws_y, P.N, s);
        }
        TFMM_CUDA_CHECK(cudaMemcpyAsync(y_host, P.d_ws_y, sizeof(float2) * P.N * R, cudaMemcpyDeviceToHost, s));
        TFMM_CUDA_CHECK(cudaStreamSynchronize(s));
    });
}

tfmm_status tfmm_planewave(const tfmm_plan* plan, const double* khat, const double* pol, int32_t R, tfmm_cfloat* V,
                           void* stream) {
    return guarded([&] {
        TFMM_REQUIRE(plan && khat && pol && V, "null argument");
        TFMM_REQUIRE(R >= 1, "R must be >= 1");
        planewave_rhs(plan->p, khat, pol, R, reinterpret_cast<float2*>(V), (cudaStream_t)stream);
    });
}

tfmm_status tfmm_translate(tfmm_plan* plan, const tfmm_cfloat* spectra_out, int32_t R, tfmm_cfloat* spectra_in,
                           void* stream) {
    return guarded([&] {
        TFMM_REQUIRE(plan, "null plan");
        TFMM_REQUIRE(spectra_out && spectra_in, "null buffer");
        TFMM_REQUIRE(spectra_out != spectra_in, "spectra_out and spectra_in must not be the same buffer");
        TFMM_REQUIRE(R >= 1 && R <= plan->p.params.max_rhs, "R must be in 1..max_rhs");
        NvtxRange nvtx("tfmm_translate");
        launch_translate(plan->p, reinterpret_cast<const float2*>(spectra_out), R, reinterpret_cast<float2*>(spectra_in),
                         (cudaStream_t)stream);
    });
}

tfmm_status tfmm_planewave_noalloc(const tfmm_plan* plan, const double* khat, const double* pol, int32_t R,
                                   tfmm_cfloat* V, void* stream) {
    return guarded([&] {
        TFMM_REQUIRE(plan && khat && pol && V, "null argument");
        planewave_rhs_noalloc(plan->p, khat, pol, R, reinterpret_cast<float2*>(V), (cudaStream_t)stream);
    });
}

}  // extern "C"
