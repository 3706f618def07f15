// Setup stage on the GPU (Sec. II.A-B): far-field tensors of every group
// (Eq. 4) in FP64, then a sequentially truncated HOSVD (Eq. 6) in FP64.
//
// Far-field: P^{alpha,+}_{n,i} = alpha_i . int b_n(r) exp(+j k k_i.(r - r_v)) dr,
// by a collapsed (Duffy) Gauss-Legendre rule on each of the two triangles of
// the RWG; alpha_i is orthogonal to k_i, so the (I - k k) projector drops out.
//
// HOSVD: the factor of each mode is the leading eigenvector block of the Gram
// matrix of that mode's unfolding (left singular vectors of the unfolding),
// truncated where the discarded energy drops to (gamma^2/3) ||A||_F^2, which is
// the per-mode gamma/sqrt(3) rule of Sec. III.A and gives ||A - A_hat||_F <=
// gamma ||A||_F.  The discarded energy is not read off the Gram's eigenvalues,
// whose absolute error is of order eps ||A||^2 (the Gram squares the condition
// number): the energy along each eigenvector v is recomputed from the unfolding
// itself, ||v^H A_(p)||^2, accurate to order eps ||A|| ||v^H A_(p)||, so tails
// far below eps ||A||^2 (gamma = 1e-8) are resolved.  The modes are processed in the order
// theta, phi, beta and each later unfolding is that of the tensor already
// projected on the earlier factors (sequential truncation; same bound as the
// plain HOSVD of ref. [26]).  For the beta mode the smaller of the two Gram
// matrices Z Z^H (n_beta) and Z^H Z (r_theta r_phi) is decomposed; in the
// second case the factor is re-orthonormalised by a Householder QR.  For the
// beta mode a range-limited eigen-solver returns only the eigenvectors above the
// truncation level while that level is well above the Gram's rounding; below
// it every eigenvector is computed and the energies come from Z as above.
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <cstdio>
#include <exception>
#include <limits>
#include <memory>
#include <mutex>
#include <thread>

#include "internal.h"

namespace tfmm {

namespace {

#define CUBLAS_CHECK(call)                                                                          \
    do {                                                                                            \
        cublasStatus_t st_ = (call);                                                                \
        if (st_ != CUBLAS_STATUS_SUCCESS)                                                           \
            fail(st_ == CUBLAS_STATUS_ALLOC_FAILED ? TFMM_OOM : TFMM_CUDA,                          \
                 std::string(#call) + " failed with cuBLAS status " + std::to_string((int)st_));   \
    } while (0)

#define CUSOLVER_CHECK(call)                                                                        \
    do {                                                                                            \
        cusolverStatus_t st_ = (call);                                                              \
        if (st_ != CUSOLVER_STATUS_SUCCESS)                                                         \
            fail(st_ == CUSOLVER_STATUS_ALLOC_FAILED ? TFMM_OOM : TFMM_CUDA,                        \
                 std::string(#call) + " failed with cuSOLVER status " + std::to_string((int)st_)); \
    } while (0)

constexpr int kMaxQuad = 10;  // collapsed rule order cap: 100 points per triangle
__constant__ double c_qu[kMaxQuad * kMaxQuad];
__constant__ double c_qv[kMaxQuad * kMaxQuad];
__constant__ double c_qw[kMaxQuad * kMaxQuad];

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    explicit DevBuf(size_t b) { alloc(b); }
    void alloc(size_t b) {
        release();
        if (b == 0) return;
        TFMM_CUDA_CHECK(device_malloc(&p, b));
        bytes = b;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    ~DevBuf() { release(); }
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

// --------------------------------------------------------------- far-field
constexpr int kFFThreads = 128;  // directions per block
constexpr int kFFRwgs = 4;       // RWGs per block

struct FFArgs {
    const RwgGeom* geom;      // global RWG order
    const int* grp_rwg;       // RWG ids, group order
    const int64_t* rwg_off;   // per batch group: offset into grp_rwg
    const int* nbeta;         // per batch group
    const int64_t* out_off;   // per batch group: offset (double2) of its [alpha][n][i] block
    const double* centre;     // per batch group, 3
    const double* dirs;       // n_dir x 9: k_hat, theta_hat, phi_hat
    double2* out;
    double k;
    int n_dir, nq;            // nq points per triangle
};

__global__ void __launch_bounds__(kFFThreads) farfield_kernel(const FFArgs a) {
    __shared__ double s_pt[kFFRwgs][2 * kMaxQuad * kMaxQuad][3];
    __shared__ double s_am[kFFRwgs][2 * kMaxQuad * kMaxQuad][3];
    const int gb = blockIdx.z;
    const int nb = a.nbeta[gb];
    const int n0 = blockIdx.y * kFFRwgs;
    if (n0 >= nb) return;
    const int nr = min(kFFRwgs, nb - n0);
    const double cx = a.centre[3 * gb], cy = a.centre[3 * gb + 1], cz = a.centre[3 * gb + 2];
    const int npts = 2 * a.nq;
    // quadrature points (relative to the box centre) and vector amplitudes
    for (int e = threadIdx.x; e < nr * npts; e += blockDim.x) {
        const int rr = e / npts, q = e % npts;
        const RwgGeom g = a.geom[a.grp_rwg[a.rwg_off[gb] + n0 + rr]];
        const int side = q >= a.nq;
        const int qq = side ? q - a.nq : q;
        const double* p = side ? g.pm : g.pp;
        const double u = c_qu[qq], v = c_qv[qq], w = c_qw[qq];
        const double sgn = side ? -1.0 : 1.0;
        double r[3];
        for (int c = 0; c < 3; ++c) {
            r[c] = p[c] + u * (g.q1[c] - p[c]) + v * (1.0 - u) * (g.q2[c] - p[c]);
            s_am[rr][q][c] = sgn * g.l * w * (r[c] - p[c]);
        }
        s_pt[rr][q][0] = r[0] - cx;
        s_pt[rr][q][1] = r[1] - cy;
        s_pt[rr][q][2] = r[2] - cz;
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_dir) return;
    const double* d = a.dirs + 9 * (int64_t)i;
    const double kx = a.k * d[0], ky = a.k * d[1], kz = a.k * d[2];
    for (int rr = 0; rr < nr; ++rr) {
        double jr[3] = {0, 0, 0}, ji[3] = {0, 0, 0};
        for (int q = 0; q < npts; ++q) {
            const double psi = kx * s_pt[rr][q][0] + ky * s_pt[rr][q][1] + kz * s_pt[rr][q][2];
            double sn, cs;
            sincos(psi, &sn, &cs);
            for (int c = 0; c < 3; ++c) {
                jr[c] += s_am[rr][q][c] * cs;
                ji[c] += s_am[rr][q][c] * sn;
            }
        }
        const int n = n0 + rr;
        double2* o = a.out + a.out_off[gb];
        double2 pt, pp;
        pt.x = d[3] * jr[0] + d[4] * jr[1] + d[5] * jr[2];
        pt.y = d[3] * ji[0] + d[4] * ji[1] + d[5] * ji[2];
        pp.x = d[6] * jr[0] + d[7] * jr[1] + d[8] * jr[2];
        pp.y = d[6] * ji[0] + d[7] * ji[1] + d[8] * ji[2];
        o[(int64_t)n * a.n_dir + i] = pt;
        o[(int64_t)nb * a.n_dir + (int64_t)n * a.n_dir + i] = pp;
    }
}

// ------------------------------------------------------------ small kernels
// out[perm] of a 3-D column-major array in[i0 + d0 (i1 + d1 i2)].
// mode 0: out[i0 + d0 (i2 + d2 i1)]  (swap the last two indices)
// mode 1: out[i1 + d1 (i0 + d0 i2)]  (swap the first two indices)
__global__ void permute3_kernel(const double2* __restrict__ in, double2* __restrict__ out, int d0, int d1,
                                int d2, int mode) {
    const int64_t total = (int64_t)d0 * d1 * d2;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i0 = (int)(e % d0);
        const int64_t rest = e / d0;
        const int i1 = (int)(rest % d1);
        const int i2 = (int)(rest / d1);
        int64_t o;
        if (mode == 0)
            o = i0 + (int64_t)d0 * (i2 + (int64_t)d2 * i1);
        else
            o = i1 + (int64_t)d1 * (i0 + (int64_t)d0 * i2);
        out[o] = in[e];
    }
}

// out (n x r, ld n) = rows 0..n-1 of columns lastcol, lastcol-1, ... of G (ld ldg),
// i.e. the eigenvectors of the r largest eigenvalues, largest first; conj optional.
__global__ void take_top_kernel(const double2* __restrict__ G, int ldg, int n, int lastcol, int r,
                                double2* __restrict__ out, int conj_out) {
    const int64_t total = (int64_t)n * r;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), j = (int)(e / n);
        double2 v = G[i + (int64_t)ldg * (lastcol - j)];
        if (conj_out) v.y = -v.y;
        out[e] = v;
    }
}

// FP64 -> FP32 copy of an n x m column-major block into a buffer with leading dimension ldo.
__global__ void to_f32_kernel(const double2* __restrict__ in, int64_t n, int64_t m, int64_t ldi,
                              float2* __restrict__ out, int64_t ldo) {
    const int64_t total = n * m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % n, j = e / n;
        const double2 v = in[i + ldi * j];
        out[i + ldo * j] = make_float2((float)v.x, (float)v.y);
    }
}

// --------------------------------------------------------- plane-wave RHS
struct PWArgs {
    const RwgGeom* geom;
    const double* khat;  // R x 3
    const double* pol;   // R x 3
    float2* V;
    double k;
    int64_t n;
    int R, nq;
};

__global__ void planewave_kernel(const PWArgs a) {
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (m >= a.n) return;
    const RwgGeom g = a.geom[m];
    const double* kh = a.khat + 3 * r;
    const double* p = a.pol + 3 * r;
    double vr = 0.0, vi = 0.0;
    for (int side = 0; side < 2; ++side) {
        const double* pv = side ? g.pm : g.pp;
        const double sgn = side ? -1.0 : 1.0;
        for (int q = 0; q < a.nq; ++q) {
            const double u = c_qu[q], v = c_qv[q], w = c_qw[q];
            double r3[3], dot = 0.0, ph = 0.0;
            for (int c = 0; c < 3; ++c) {
                r3[c] = pv[c] + u * (g.q1[c] - pv[c]) + v * (1.0 - u) * (g.q2[c] - pv[c]);
                dot += sgn * g.l * w * (r3[c] - pv[c]) * p[c];
                ph += kh[c] * r3[c];
            }
            double sn, cs;
            sincos(-a.k * ph, &sn, &cs);
            vr -= dot * cs;
            vi -= dot * sn;
        }
    }
    a.V[m + a.n * r] = make_float2((float)vr, (float)vi);
}

int grid1d(int64_t total, int threads = 256) {
    int64_t b = (total + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 65535 * 8));
}

void upload_quadrature(int order, cudaStream_t s) {
    std::vector<double> x, w;
    gauss_legendre(order, x, w);
    std::vector<double> qu, qv, qw;
    for (int a = 0; a < order; ++a)
        for (int b = 0; b < order; ++b) {
            const double u = 0.5 * (x[a] + 1.0), v = 0.5 * (x[b] + 1.0);
            qu.push_back(u);
            qv.push_back(v);
            qw.push_back(0.25 * w[a] * w[b] * (1.0 - u));  // sum = 1/2: int_T f = 2A sum w f
        }
    TFMM_CUDA_CHECK(cudaMemcpyToSymbolAsync(c_qu, qu.data(), qu.size() * sizeof(double), 0,
                                            cudaMemcpyHostToDevice, s));
    TFMM_CUDA_CHECK(cudaMemcpyToSymbolAsync(c_qv, qv.data(), qv.size() * sizeof(double), 0,
                                            cudaMemcpyHostToDevice, s));
    TFMM_CUDA_CHECK(cudaMemcpyToSymbolAsync(c_qw, qw.data(), qw.size() * sizeof(double), 0,
                                            cudaMemcpyHostToDevice, s));
}

std::vector<double> direction_table(const Plan& P) {
    std::vector<double> dirs((size_t)P.n_dir * 9);
    for (int ip = 0; ip < P.n_phi; ++ip)
        for (int it = 0; it < P.n_theta; ++it) {
            const double t = P.theta[it], ph = P.phi[ip];
            const double st = std::sin(t), ct = std::cos(t), sp = std::sin(ph), cp = std::cos(ph);
            double* d = &dirs[9 * ((size_t)it + (size_t)P.n_theta * ip)];
            d[0] = st * cp; d[1] = st * sp; d[2] = ct;
            d[3] = ct * cp; d[4] = ct * sp; d[5] = -st;
            d[6] = -sp;     d[7] = cp;      d[8] = 0.0;
        }
    return dirs;
}

double ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// Smallest r >= 1 whose discarded eigenvalues (ascending list, clamped at 0) sum to <= thr2;
// tail0 is energy already discarded outside the list.
int choose_rank(const double* ev, int n, double thr2, double tail0 = 0.0) {
    double tail = tail0;
    if (tail > thr2) return std::max(n, 1);
    int r = n;
    for (int i = 0; i < n; ++i) {  // discard i+1 smallest
        tail += std::max(ev[i], 0.0);
        if (tail <= thr2 && n - (i + 1) >= 1)
            r = n - (i + 1);
        else
            break;
    }
    return std::max(r, 1);
}

// Batched Hermitian eigen-decomposition of `count` n x n matrices (lower part
// valid, ld n, stride n*n) with eigenvalues ascending in W (count x n): the
// batched cuSOLVER solver when the library accepts the size, else one Xsyevd
// per matrix (TFMM_EIG=single forces the latter).
void eig_batched(cusolverDnHandle_t sol, cusolverDnParams_t prm, double2* A, double* W, int n, int count,
                 cudaStream_t s) {
    if (count == 0) return;
    const char* env = std::getenv("TFMM_EIG");
    size_t dbytes = 0, hbytes = 0;
    DevBuf info(sizeof(int) * count);
    const bool force_single = env && std::strcmp(env, "single") == 0;
    cusolverStatus_t st = CUSOLVER_STATUS_NOT_SUPPORTED;
    if (!force_single)
        st = cusolverDnXsyevBatched_bufferSize(sol, prm, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n,
                                               CUDA_C_64F, A, n, CUDA_R_64F, W, CUDA_C_64F, &dbytes, &hbytes, count);
    if (st == CUSOLVER_STATUS_SUCCESS) {
        DevBuf work(std::max<size_t>(dbytes, 16));
        std::vector<char> hwork(std::max<size_t>(hbytes, 16));
        CUSOLVER_CHECK(cusolverDnXsyevBatched(sol, prm, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n,
                                              CUDA_C_64F, A, n, CUDA_R_64F, W, CUDA_C_64F, work.p, dbytes,
                                              hwork.data(), hbytes, info.as<int>(), count));
    } else {
        CUSOLVER_CHECK(cusolverDnXsyevd_bufferSize(sol, prm, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n,
                                                   CUDA_C_64F, A, n, CUDA_R_64F, W, CUDA_C_64F, &dbytes, &hbytes));
        DevBuf work(std::max<size_t>(dbytes, 16));
        std::vector<char> hwork(std::max<size_t>(hbytes, 16));
        for (int i = 0; i < count; ++i)
            CUSOLVER_CHECK(cusolverDnXsyevd(sol, prm, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, CUDA_C_64F,
                                            A + (int64_t)i * n * n, n, CUDA_R_64F, W + (int64_t)i * n, CUDA_C_64F,
                                            work.p, dbytes, hwork.data(), hbytes, info.as<int>() + i));
    }
    std::vector<int> hinfo(count);
    TFMM_CUDA_CHECK(cudaMemcpyAsync(hinfo.data(), info.p, sizeof(int) * count, cudaMemcpyDeviceToHost, s));
    TFMM_CUDA_CHECK(cudaStreamSynchronize(s));
    for (int i = 0; i < count; ++i)
        if (hinfo[i] != 0) fail(TFMM_NUMERIC, "eigen-decomposition failed (info " + std::to_string(hinfo[i]) + ")");
}

// out[e] = sum over parts of part[j][e] (FP64 complex), e < count
__global__ void sum_parts_kernel(const double2* __restrict__ part, int nparts, int64_t count, double2* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        for (int j = 0; j < nparts; ++j) {
            const double2 v = part[(int64_t)j * count + e];
            acc.x += v.x;
            acc.y += v.y;
        }
        out[e] = acc;
    }
}

// count n x n column-reversed identity matrices, back to back: the theta / phi
// "eigenvectors" of an SVD plan, stored like an eigen-solver's output (ascending),
// so that take_top_kernel, which reads the columns from the last one back, yields
// the identity itself.
__global__ void identity_kernel(double2* __restrict__ G, int n, int count) {
    const int64_t total = (int64_t)count * n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e % ((int64_t)n * n);
        G[e] = make_double2((r % n) == n - 1 - (r / n) ? 1.0 : 0.0, 0.0);
    }
}

// out[j] = sum_{i < rows} |E[i + ld j]|^2: one block of 256 threads per column, summed in
// a fixed order (the ranks chosen from these energies do not depend on timing).
constexpr int kEnergyThreads = 256;
__global__ void __launch_bounds__(kEnergyThreads) col_energy_kernel(const double2* __restrict__ E, int64_t rows,
                                                                    int64_t ld, double* __restrict__ out) {
    __shared__ double red[kEnergyThreads];
    const int64_t j = blockIdx.x;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < rows; i += kEnergyThreads) {
        const double2 v = E[i + ld * j];
        acc += v.x * v.x + v.y * v.y;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kEnergyThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[j] = red[0];
}

struct Worker {  // one host thread's stream and library handles for per-tensor setup work
    cudaStream_t s = nullptr;
    cublasHandle_t blas = nullptr;
    cusolverDnHandle_t sol = nullptr;
    cusolverDnParams_t prm = nullptr;
    Worker() {
        TFMM_CUDA_CHECK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        CUBLAS_CHECK(cublasCreate(&blas));
        CUBLAS_CHECK(cublasSetStream(blas, s));
        CUSOLVER_CHECK(cusolverDnCreate(&sol));
        CUSOLVER_CHECK(cusolverDnSetStream(sol, s));
        CUSOLVER_CHECK(cusolverDnCreateParams(&prm));
    }
    ~Worker() {
        if (prm) cusolverDnDestroyParams(prm);
        if (sol) cusolverDnDestroy(sol);
        if (blas) cublasDestroy(blas);
        if (s) cudaStreamDestroy(s);
    }
    Worker(const Worker&) = delete;
    Worker& operator=(const Worker&) = delete;
};

struct Timers {
    double mode1 = 0, mode2 = 0, gram3 = 0, eig3 = 0, fac3 = 0;
};

// Runs f(worker, i) for i in [0, n) on the worker threads (round robin), each
// thread on the caller's device; rethrows the first failure.
template <class F>
void parallel_for(std::vector<std::unique_ptr<Worker>>& pool, int n, F&& f) {
    int dev = 0;
    TFMM_CUDA_CHECK(cudaGetDevice(&dev));
    const int nw = (int)pool.size();
    std::vector<std::exception_ptr> errs(nw);
    std::vector<std::thread> th;
    for (int w = 0; w < nw; ++w)
        th.emplace_back([&, w] {
            try {
                TFMM_CUDA_CHECK(cudaSetDevice(dev));
                for (int i = w; i < n; i += nw) f(*pool[w], w, i);
                TFMM_CUDA_CHECK(cudaStreamSynchronize(pool[w]->s));
            } catch (...) {
                errs[w] = std::current_exception();
            }
        });
    for (auto& t : th) t.join();
    for (auto& e : errs)
        if (e) std::rethrow_exception(e);
}

// One Hermitian eigen-decomposition (lower part valid, in place, eigenvalues ascending).
void eig_one(Worker& w, double2* A, double* W, int n, int* info) {
    size_t dbytes = 0, hbytes = 0;
    CUSOLVER_CHECK(cusolverDnXsyevd_bufferSize(w.sol, w.prm, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n,
                                               CUDA_C_64F, A, n, CUDA_R_64F, W, CUDA_C_64F, &dbytes, &hbytes));
    DevBuf work(std::max<size_t>(dbytes, 16));
    std::vector<char> hwork(std::max<size_t>(hbytes, 16));
    CUSOLVER_CHECK(cusolverDnXsyevd(w.sol, w.prm, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, CUDA_C_64F, A,
                                    n, CUDA_R_64F, W, CUDA_C_64F, work.p, dbytes, hwork.data(), hbytes, info));
    int h = 0;
    TFMM_CUDA_CHECK(cudaMemcpyAsync(&h, info, sizeof(int), cudaMemcpyDeviceToHost, w.s));
    TFMM_CUDA_CHECK(cudaStreamSynchronize(w.s));  // the workspaces above are released on return
    if (h != 0) fail(TFMM_NUMERIC, "eigen-decomposition failed (info " + std::to_string(h) + ")");
}

constexpr int kGramParts = 64;

// Gram matrix of a short, wide operand by split-K: the long dimension is cut
// into chunks, one strided-batched ZGEMM forms a partial Gram per chunk and a
// reduction sums them (cuBLAS ZHERK parallelises such shapes poorly).
//   rows = true : G = A A^H, A is n x k column-major (ld lda)
//   rows = false: G = A^H A, A is k x n column-major (ld lda)
// part: scratch of at least (kGramParts + 1) n^2 elements.  G is n x n, both triangles.
void gram_splitk(Worker& w, bool rows, int n, int64_t k, const double2* A, int64_t lda, double2* G, double2* part) {
    const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
    const int64_t kc = std::max<int64_t>(128, (k + kGramParts - 1) / kGramParts);
    const int nfull = (int)(k / kc);
    const int64_t krem = k - (int64_t)nfull * kc;
    const int64_t nn = (int64_t)n * n;
    const cublasOperation_t oa = rows ? CUBLAS_OP_N : CUBLAS_OP_C, ob = rows ? CUBLAS_OP_C : CUBLAS_OP_N;
    const int64_t stride = rows ? lda * kc : kc;
    if (nfull > 0)
        CUBLAS_CHECK(cublasZgemmStridedBatched(w.blas, oa, ob, n, n, (int)kc, &one, (const cuDoubleComplex*)A, (int)lda,
                                               stride, (const cuDoubleComplex*)A, (int)lda, stride, &zero,
                                               (cuDoubleComplex*)part, n, nn, nfull));
    int nparts = nfull;
    if (krem > 0) {
        const double2* Ar = A + (rows ? lda * kc * nfull : kc * nfull);
        CUBLAS_CHECK(cublasZgemm(w.blas, oa, ob, n, n, (int)krem, &one, (const cuDoubleComplex*)Ar, (int)lda,
                                 (const cuDoubleComplex*)Ar, (int)lda, &zero, (cuDoubleComplex*)(part + nn * nfull),
                                 n));
        ++nparts;
    }
    sum_parts_kernel<<<grid1d(nn), 256, 0, w.s>>>(part, nparts, nn, G);
    TFMM_CUDA_CHECK(cudaGetLastError());
}

struct Tensor {      // one (group, alpha) tensor of the current batch
    int g, alpha, nb;
    double2* A;      // n_theta x n_phi x nb
    double norm2 = 0;  // ||A||_F^2
    double z2 = 0;     // energy left after the theta and phi projections
    int rt = 0, rp = 0, rb = 0;
};

// Sequentially truncated HOSVD of every tensor of a batch (modes theta, phi, beta).
void hosvd_batch(Plan& P, std::vector<Tensor>& T, std::vector<std::unique_ptr<Worker>>& pool, cudaStream_t s,
                 Timers& tm) {
    (void)s;
    const int nt = P.n_theta, np = P.n_phi;
    const int nT = (int)T.size();
    const int nw = (int)pool.size();
    // Tucker: gamma / sqrt(3) per mode (Sec. III.A).  SVD (Sec. II.C comparator): the theta
    // and phi modes are kept whole (identity factors) and the beta mode, whose unfolding is
    // the transposed aggregation matrix, is truncated at gamma itself (note under Table II).
    const bool svd = plan_is_svd(P);
    const double tol2 = P.params.tol * P.params.tol / 3.0;
    const double tol2_beta = svd ? P.params.tol * P.params.tol : tol2;
    const double r_one = 1.0, r_zero = 0.0;
    const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
    const char* env = std::getenv("TFMM_EIG");
    const bool batched_small = !(env && std::strcmp(env, "single") == 0);
    auto t0 = std::chrono::steady_clock::now();
    std::vector<DevBuf> winfo(nw);
    for (auto& b : winfo) b.alloc(sizeof(int));

    // mode theta: G1 = A_(1) A_(1)^H (n_theta x n_theta)
    DevBuf d_G1(sizeof(double2) * nT * nt * nt), d_W1(sizeof(double) * nT * nt);
    const int ngmax = std::max(nt, np);
    std::vector<DevBuf> wpart(nw);
    for (auto& b : wpart) b.alloc(sizeof(double2) * (int64_t)(kGramParts + 1) * ngmax * ngmax);
    if (svd) {
        Worker& w0 = *pool[0];
        identity_kernel<<<grid1d((int64_t)nT * nt * nt), 256, 0, w0.s>>>(d_G1.as<double2>(), nt, nT);
        TFMM_CUDA_CHECK(cudaGetLastError());
        TFMM_CUDA_CHECK(cudaStreamSynchronize(w0.s));
    } else {
        parallel_for(pool, nT, [&](Worker& w, int wi, int t) {
            gram_splitk(w, true, nt, (int64_t)np * T[t].nb, T[t].A, nt, d_G1.as<double2>() + (int64_t)t * nt * nt,
                        wpart[wi].as<double2>());
            if (!batched_small)
                eig_one(w, d_G1.as<double2>() + (int64_t)t * nt * nt, d_W1.as<double>() + (int64_t)t * nt, nt,
                        winfo[wi].as<int>());
        });
        if (batched_small) {
            Worker& w0 = *pool[0];
            eig_batched(w0.sol, w0.prm, d_G1.as<double2>(), d_W1.as<double>(), nt, nT, w0.s);
        }
    }
    // Energy of the unfolding along every eigenvector, e_i = ||v_i^H A_(1)||^2, from the
    // unfolding itself: the Gram's eigenvalues carry absolute errors of order eps ||A||^2,
    // while these are accurate to order eps ||A|| ||v_i^H A_(1)||, which resolves tails far
    // below eps ||A||^2 (tolerances near 1e-8).  The ranks are chosen from them.
    int maxnb = 1;
    for (int t = 0; t < nT; ++t) maxnb = std::max(maxnb, T[t].nb);
    std::vector<DevBuf> wA(nw);
    for (auto& b : wA) b.alloc(sizeof(double2) * (int64_t)nt * np * maxnb);
    DevBuf d_E1(sizeof(double) * nT * nt);
    parallel_for(pool, nT, [&](Worker& w, int wi, int t) {
        // A_(1)^H V (n_phi n_beta x n_theta): elementwise the modulus of V^H A_(1)
        const int64_t cols = (int64_t)np * T[t].nb;
        CUBLAS_CHECK(cublasZgemm(w.blas, CUBLAS_OP_C, CUBLAS_OP_N, (int)cols, nt, nt, &one,
                                 (const cuDoubleComplex*)T[t].A, nt,
                                 (const cuDoubleComplex*)(d_G1.as<double2>() + (int64_t)t * nt * nt), nt, &zero,
                                 (cuDoubleComplex*)wA[wi].p, (int)cols));
        col_energy_kernel<<<nt, kEnergyThreads, 0, w.s>>>(wA[wi].as<double2>(), cols, cols,
                                                          d_E1.as<double>() + (int64_t)t * nt);
        TFMM_CUDA_CHECK(cudaGetLastError());
    });
    std::vector<double> E1((size_t)nT * nt);
    TFMM_CUDA_CHECK(cudaMemcpy(E1.data(), d_E1.p, sizeof(double) * E1.size(), cudaMemcpyDeviceToHost));
    int64_t y1_tot = 0;
    std::vector<int64_t> y1_off(nT);
    for (int t = 0; t < nT; ++t) {
        double n2 = 0;
        for (int i = 0; i < nt; ++i) n2 += E1[(size_t)t * nt + i];
        T[t].norm2 = n2;
        T[t].rt = svd ? nt : choose_rank(&E1[(size_t)t * nt], nt, tol2 * n2);
        y1_off[t] = y1_tot;
        y1_tot += (int64_t)T[t].rt * np * T[t].nb;
    }
    tm.mode1 += ms_since(t0);
    t0 = std::chrono::steady_clock::now();

    // U_theta; A1 = U_theta^H A_(1) -> [a, i_phi, n]; Y1 = [a, n, i_phi]; G2' = Y1^H Y1
    DevBuf d_Ut(sizeof(double2) * nT * nt * nt), d_Y1(sizeof(double2) * std::max<int64_t>(y1_tot, 1));
    DevBuf d_G2(sizeof(double2) * nT * np * np), d_W2(sizeof(double) * nT * np);
    parallel_for(pool, nT, [&](Worker& w, int wi, int t) {
        const int rt = T[t].rt, nb = T[t].nb;
        double2* Ut = d_Ut.as<double2>() + (int64_t)t * nt * nt;
        take_top_kernel<<<grid1d((int64_t)nt * rt), 256, 0, w.s>>>(d_G1.as<double2>() + (int64_t)t * nt * nt, nt, nt,
                                                                     nt - 1, rt, Ut, 0);
        CUBLAS_CHECK(cublasZgemm(w.blas, CUBLAS_OP_C, CUBLAS_OP_N, rt, np * nb, nt, &one, (const cuDoubleComplex*)Ut, nt,
                                 (const cuDoubleComplex*)T[t].A, nt, &zero, (cuDoubleComplex*)wA[wi].p, rt));
        permute3_kernel<<<grid1d((int64_t)rt * np * nb), 256, 0, w.s>>>(wA[wi].as<double2>(),
                                                                         d_Y1.as<double2>() + y1_off[t], rt, np, nb, 0);
        TFMM_CUDA_CHECK(cudaGetLastError());
        if (svd) {
            identity_kernel<<<grid1d((int64_t)np * np), 256, 0, w.s>>>(d_G2.as<double2>() + (int64_t)t * np * np, np, 1);
            TFMM_CUDA_CHECK(cudaGetLastError());
            return;
        }
        gram_splitk(w, false, np, (int64_t)rt * nb, d_Y1.as<double2>() + y1_off[t], (int64_t)rt * nb,
                    d_G2.as<double2>() + (int64_t)t * np * np, wpart[wi].as<double2>());
        if (!batched_small)
            eig_one(w, d_G2.as<double2>() + (int64_t)t * np * np, d_W2.as<double>() + (int64_t)t * np, np,
                    winfo[wi].as<int>());
    });
    if (batched_small && !svd) {
        Worker& w0 = *pool[0];
        eig_batched(w0.sol, w0.prm, d_G2.as<double2>(), d_W2.as<double>(), np, nT, w0.s);
    }
    // energies e_j = ||Y1 v_j||^2 of the theta-projected unfolding along every eigenvector
    DevBuf d_E2(sizeof(double) * nT * np);
    parallel_for(pool, nT, [&](Worker& w, int wi, int t) {
        const int64_t rows = (int64_t)T[t].rt * T[t].nb;
        CUBLAS_CHECK(cublasZgemm(w.blas, CUBLAS_OP_N, CUBLAS_OP_N, (int)rows, np, np, &one,
                                 (const cuDoubleComplex*)(d_Y1.as<double2>() + y1_off[t]), (int)rows,
                                 (const cuDoubleComplex*)(d_G2.as<double2>() + (int64_t)t * np * np), np, &zero,
                                 (cuDoubleComplex*)wA[wi].p, (int)rows));
        col_energy_kernel<<<np, kEnergyThreads, 0, w.s>>>(wA[wi].as<double2>(), rows, rows,
                                                          d_E2.as<double>() + (int64_t)t * np);
        TFMM_CUDA_CHECK(cudaGetLastError());
    });
    std::vector<double> E2((size_t)nT * np);
    TFMM_CUDA_CHECK(cudaMemcpy(E2.data(), d_E2.p, sizeof(double) * E2.size(), cudaMemcpyDeviceToHost));
    int n3max = 1, mmax = 1;
    for (int t = 0; t < nT; ++t) {
        T[t].rp = svd ? np : choose_rank(&E2[(size_t)t * np], np, tol2 * T[t].norm2);
        double z2 = 0.0;
        for (int i = np - T[t].rp; i < np; ++i) z2 += E2[(size_t)t * np + i];
        T[t].z2 = z2;
        mmax = std::max(mmax, T[t].rt * T[t].rp);
        n3max = std::max(n3max, std::min(T[t].nb, T[t].rt * T[t].rp));
    }
    tm.mode2 += ms_since(t0);
    t0 = std::chrono::steady_clock::now();
    std::vector<DevBuf> wV(nw);
    for (auto& b : wV) b.alloc(sizeof(double2) * (int64_t)std::max(np, mmax) * std::max(np, n3max));

    // mode beta, in two passes over the batch.  Pass A (per tensor): Z = [n, a, b]
    // (n_beta x m, m = r_t r_p), Gram of its smaller side, eigen-decomposition, rank.
    // Then one allocation holds the batch's FP64 factors.  Pass B (per tensor):
    // U_beta (QR-orthonormalised when taken from Z V), core C_(3) = U_beta^H Z.
    int64_t z_tot = 0, g3_tot = 0;
    std::vector<int64_t> z_off(nT), g3_off(nT);
    for (int t = 0; t < nT; ++t) {
        const int m = T[t].rt * T[t].rp, n = std::min(T[t].nb, m);
        z_off[t] = z_tot;
        z_tot += (int64_t)T[t].nb * m;
        g3_off[t] = g3_tot;
        g3_tot += (int64_t)n * n;
    }
    DevBuf d_Z(sizeof(double2) * std::max<int64_t>(z_tot, 1)), d_G3(sizeof(double2) * std::max<int64_t>(g3_tot, 1));
    DevBuf d_W3(sizeof(double) * std::max<int64_t>((int64_t)nT * n3max, 1));
    // eigen-solver workspace per worker, sized for the largest problem of the batch
    // default: Xsyevdx, eigenvectors only for eigenvalues above (gamma^2/6 ||A||^2) / n, whose
    // sum bounds what it leaves out by half the truncation budget; TFMM_EIG3=syevd: all of them
    const char* e3 = std::getenv("TFMM_EIG3");
    const bool use_dx = !(e3 && std::strcmp(e3, "syevd") == 0);
    size_t eig_d = 16, eig_h = 16;
    {
        Worker& w0 = *pool[0];
        for (int t = 0; t < nT; ++t) {
            const int n = std::min(T[t].nb, T[t].rt * T[t].rp);
            size_t db = 0, hb = 0;
            CUSOLVER_CHECK(cusolverDnXsyevd_bufferSize(w0.sol, w0.prm, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER,
                                                       n, CUDA_C_64F, d_G3.p, n, CUDA_R_64F, d_W3.p, CUDA_C_64F, &db,
                                                       &hb));
            eig_d = std::max(eig_d, db);
            eig_h = std::max(eig_h, hb);
            if (use_dx) {
                double vl = 0.0, vu = 1.0;
                int64_t meig = 0;
                CUSOLVER_CHECK(cusolverDnXsyevdx_bufferSize(w0.sol, w0.prm, CUSOLVER_EIG_MODE_VECTOR,
                                                            CUSOLVER_EIG_RANGE_V, CUBLAS_FILL_MODE_LOWER, n, CUDA_C_64F,
                                                            d_G3.p, n, &vl, &vu, 0, 0, &meig, CUDA_R_64F, d_W3.p,
                                                            CUDA_C_64F, &db, &hb));
                eig_d = std::max(eig_d, db);
                eig_h = std::max(eig_h, hb);
            }
        }
    }
    std::vector<DevBuf> weig(nw);
    std::vector<std::vector<char>> weigh(nw);
    for (int i = 0; i < nw; ++i) {
        weig[i].alloc(eig_d);
        weigh[i].resize(eig_h);
    }
    std::vector<double> ms_g(nw, 0.0), ms_e(nw, 0.0), ms_f(nw, 0.0);
    std::vector<DevBuf> we3(nw);
    for (auto& b : we3) b.alloc(sizeof(double) * n3max);
    std::vector<std::vector<double>> W3(nT);
    std::vector<int> nvec(nT, 0);  // eigenvectors returned per tensor (ascending, first columns)
    parallel_for(pool, nT, [&](Worker& w, int wi, int t) {
        auto ta = std::chrono::steady_clock::now();
        const int rt = T[t].rt, rp = T[t].rp, nb = T[t].nb, m = rt * rp, n = std::min(nb, m);
        double2* Vp = wV[wi].as<double2>();
        // V_r (n_phi x r_p) from the mode-2 Gram; A2 = Y1 V_r -> [a, n, b]; Z = [n, a, b]
        take_top_kernel<<<grid1d((int64_t)np * rp), 256, 0, w.s>>>(d_G2.as<double2>() + (int64_t)t * np * np, np, np,
                                                                     np - 1, rp, Vp, 0);
        CUBLAS_CHECK(cublasZgemm(w.blas, CUBLAS_OP_N, CUBLAS_OP_N, rt * nb, rp, np, &one,
                                 (const cuDoubleComplex*)(d_Y1.as<double2>() + y1_off[t]), rt * nb,
                                 (const cuDoubleComplex*)Vp, np, &zero, (cuDoubleComplex*)wA[wi].p, rt * nb));
        double2* Z = d_Z.as<double2>() + z_off[t];
        permute3_kernel<<<grid1d((int64_t)rt * nb * rp), 256, 0, w.s>>>(wA[wi].as<double2>(), Z, rt, nb, rp, 1);
        TFMM_CUDA_CHECK(cudaGetLastError());
        double2* G3 = d_G3.as<double2>() + g3_off[t];
        if (nb <= m)
            CUBLAS_CHECK(cublasZherk(w.blas, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N, nb, m, &r_one,
                                     (const cuDoubleComplex*)Z, nb, &r_zero, (cuDoubleComplex*)G3, nb));
        else
            CUBLAS_CHECK(cublasZherk(w.blas, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_C, m, nb, &r_one,
                                     (const cuDoubleComplex*)Z, nb, &r_zero, (cuDoubleComplex*)G3, m));
        auto tb = std::chrono::steady_clock::now();
        ms_g[wi] += std::chrono::duration<double, std::milli>(tb - ta).count();
        double* Wt = d_W3.as<double>() + (int64_t)t * n3max;
        const double thr2 = tol2_beta * T[t].norm2;
        // The Gram's eigenvalues resolve discarded energies only down to about eps ||Z||^2 (and
        // the energy a range-limited solve leaves out is a difference of two such numbers).
        // When the budget comes within 1000 rounding units of ||Z||^2, decompose fully and take
        // the energy along each eigenvector from Z itself, as in the theta and phi modes.
        const bool accurate = thr2 > 0.0 && thr2 < 1e3 * std::numeric_limits<double>::epsilon() * T[t].z2;
        int meig = n;
        if (use_dx && thr2 > 0.0 && !accurate) {
            double vl = 0.5 * thr2 / n, vu = 2.0 * T[t].z2 + 1.0;
            int64_t meig64 = 0;
            CUSOLVER_CHECK(cusolverDnXsyevdx(w.sol, w.prm, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_V,
                                             CUBLAS_FILL_MODE_LOWER, n, CUDA_C_64F, G3, n, &vl, &vu, 0, 0, &meig64,
                                             CUDA_R_64F, Wt, CUDA_C_64F, weig[wi].p, eig_d, weigh[wi].data(), eig_h,
                                             winfo[wi].as<int>()));
            meig = (int)meig64;
        } else {
            CUSOLVER_CHECK(cusolverDnXsyevd(w.sol, w.prm, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n,
                                            CUDA_C_64F, G3, n, CUDA_R_64F, Wt, CUDA_C_64F, weig[wi].p, eig_d,
                                            weigh[wi].data(), eig_h, winfo[wi].as<int>()));
        }
        int hinfo = 0;
        W3[t].resize(std::max(meig, 0));
        if (meig > 0)
            TFMM_CUDA_CHECK(cudaMemcpyAsync(W3[t].data(), Wt, sizeof(double) * meig, cudaMemcpyDeviceToHost, w.s));
        TFMM_CUDA_CHECK(cudaMemcpyAsync(&hinfo, winfo[wi].p, sizeof(int), cudaMemcpyDeviceToHost, w.s));
        TFMM_CUDA_CHECK(cudaStreamSynchronize(w.s));
        if (hinfo != 0) fail(TFMM_NUMERIC, "eigen-decomposition failed (info " + std::to_string(hinfo) + ")");
        if (meig < 1) fail(TFMM_NUMERIC, "no eigenvalue above the truncation bound (zero far-field tensor?)");
        if (accurate) {
            // e_i: column norms of Z^H V (left eigenvectors, n_beta <= m) or of Z V (right ones)
            double2* E = wA[wi].as<double2>();
            if (nb <= m) {
                CUBLAS_CHECK(cublasZgemm(w.blas, CUBLAS_OP_C, CUBLAS_OP_N, m, nb, nb, &one, (const cuDoubleComplex*)Z,
                                         nb, (const cuDoubleComplex*)G3, nb, &zero, (cuDoubleComplex*)E, m));
                col_energy_kernel<<<nb, kEnergyThreads, 0, w.s>>>(E, m, m, we3[wi].as<double>());
            } else {
                CUBLAS_CHECK(cublasZgemm(w.blas, CUBLAS_OP_N, CUBLAS_OP_N, nb, m, m, &one, (const cuDoubleComplex*)Z,
                                         nb, (const cuDoubleComplex*)G3, m, &zero, (cuDoubleComplex*)E, nb));
                col_energy_kernel<<<m, kEnergyThreads, 0, w.s>>>(E, nb, nb, we3[wi].as<double>());
            }
            TFMM_CUDA_CHECK(cudaGetLastError());
            TFMM_CUDA_CHECK(cudaMemcpyAsync(W3[t].data(), we3[wi].p, sizeof(double) * n, cudaMemcpyDeviceToHost, w.s));
            TFMM_CUDA_CHECK(cudaStreamSynchronize(w.s));
            T[t].rb = choose_rank(W3[t].data(), n, thr2);
        } else {
            // energy left out of the returned eigenvalues (all of it below the bound vl)
            double ret = 0.0;
            for (double v : W3[t]) ret += std::max(v, 0.0);
            const double unret = meig < n ? std::max(T[t].z2 - ret, 0.0) : 0.0;
            T[t].rb = choose_rank(W3[t].data(), meig, thr2, unret);
        }
        nvec[t] = meig;
        ms_e[wi] += ms_since(tb);
    });
    // one allocation for the batch's FP64 factors
    int64_t f_tot = 0;
    std::vector<int64_t> f_off(nT);
    int rbmax = 1;
    for (int t = 0; t < nT; ++t) {
        const int rt = T[t].rt, rp = T[t].rp, rb = T[t].rb, nb = T[t].nb;
        f_off[t] = f_tot;
        f_tot += (int64_t)nt * rt + (int64_t)np * rp + (int64_t)nb * rb + (int64_t)rt * rp * rb;
        rbmax = std::max(rbmax, rb);
    }
    double2* arena = nullptr;
    TFMM_CUDA_CHECK(device_malloc(&arena, sizeof(double2) * std::max<int64_t>(f_tot, 1)));
    P.f64_arenas.push_back(arena);
    // QR workspace per worker
    int qr_lw = 1;
    {
        Worker& w0 = *pool[0];
        for (int t = 0; t < nT; ++t) {
            const int m = T[t].rt * T[t].rp, nb = T[t].nb, rb = T[t].rb;
            if (nb <= m) continue;
            int l1 = 0, l2 = 0;
            CUSOLVER_CHECK(cusolverDnZgeqrf_bufferSize(w0.sol, nb, rb, (cuDoubleComplex*)arena, nb, &l1));
            CUSOLVER_CHECK(cusolverDnZungqr_bufferSize(w0.sol, nb, rb, rb, (cuDoubleComplex*)arena, nb,
                                                       (const cuDoubleComplex*)arena, &l2));
            qr_lw = std::max(qr_lw, std::max(l1, l2));
        }
    }
    std::vector<DevBuf> wqr(nw), wtau(nw), wC3(nw);
    for (int i = 0; i < nw; ++i) {
        wqr[i].alloc(sizeof(double2) * qr_lw);
        wtau[i].alloc(sizeof(double2) * rbmax);
        wC3[i].alloc(sizeof(double2) * (int64_t)mmax * rbmax);
    }
    parallel_for(pool, nT, [&](Worker& w, int wi, int t) {
        auto tc = std::chrono::steady_clock::now();
        const int rt = T[t].rt, rp = T[t].rp, nb = T[t].nb, m = rt * rp, rb = T[t].rb;
        HostFactors64& F = P.f64[(size_t)T[t].g * 2 + T[t].alpha];
        F.rt = rt; F.rp = rp; F.rb = rb;
        F.base = arena + f_off[t];
        const int64_t e_ut = (int64_t)nt * rt, e_up = (int64_t)np * rp, e_ub = (int64_t)nb * rb;
        double2* Ut = F.base;
        double2* Up = Ut + e_ut;
        double2* Ub = Up + e_up;
        double2* Cc = Ub + e_ub;
        const double2* Z = d_Z.as<double2>() + z_off[t];
        const double2* G3 = d_G3.as<double2>() + g3_off[t];
        double2* Vp = wV[wi].as<double2>();
        TFMM_CUDA_CHECK(cudaMemcpyAsync(Ut, d_Ut.as<double2>() + (int64_t)t * nt * nt, sizeof(double2) * e_ut,
                                        cudaMemcpyDeviceToDevice, w.s));
        // U_phi = conj(V_r)
        take_top_kernel<<<grid1d((int64_t)np * rp), 256, 0, w.s>>>(d_G2.as<double2>() + (int64_t)t * np * np, np, np,
                                                                     np - 1, rp, Up, 1);
        if (nb <= m) {
            // U_beta = leading eigenvectors of Z Z^H
            take_top_kernel<<<grid1d(e_ub), 256, 0, w.s>>>(G3, nb, nb, nvec[t] - 1, rb, Ub, 0);
        } else {
            // Q0 = Z V_r (V_r: leading eigenvectors of Z^H Z), U_beta = orthonormal basis of Q0
            take_top_kernel<<<grid1d((int64_t)m * rb), 256, 0, w.s>>>(G3, m, m, nvec[t] - 1, rb, Vp, 0);
            CUBLAS_CHECK(cublasZgemm(w.blas, CUBLAS_OP_N, CUBLAS_OP_N, nb, rb, m, &one, (const cuDoubleComplex*)Z, nb,
                                     (const cuDoubleComplex*)Vp, m, &zero, (cuDoubleComplex*)Ub, nb));
            CUSOLVER_CHECK(cusolverDnZgeqrf(w.sol, nb, rb, (cuDoubleComplex*)Ub, nb, (cuDoubleComplex*)wtau[wi].p,
                                            (cuDoubleComplex*)wqr[wi].p, qr_lw, winfo[wi].as<int>()));
            CUSOLVER_CHECK(cusolverDnZungqr(w.sol, nb, rb, rb, (cuDoubleComplex*)Ub, nb,
                                            (const cuDoubleComplex*)wtau[wi].p, (cuDoubleComplex*)wqr[wi].p, qr_lw,
                                            winfo[wi].as<int>()));
            int hinfo = 0;
            TFMM_CUDA_CHECK(cudaMemcpyAsync(&hinfo, winfo[wi].p, sizeof(int), cudaMemcpyDeviceToHost, w.s));
            TFMM_CUDA_CHECK(cudaStreamSynchronize(w.s));
            if (hinfo != 0) fail(TFMM_NUMERIC, "QR of the beta factor failed");
        }
        // core: C_(3) = U_beta^H Z (r_b x m), stored as the r_t x r_p x r_b tensor (m x r_b)
        CUBLAS_CHECK(cublasZgemm(w.blas, CUBLAS_OP_C, CUBLAS_OP_N, rb, m, nb, &one, (const cuDoubleComplex*)Ub, nb,
                                 (const cuDoubleComplex*)Z, nb, &zero, (cuDoubleComplex*)wC3[wi].p, rb));
        CUBLAS_CHECK(cublasZgeam(w.blas, CUBLAS_OP_T, CUBLAS_OP_T, m, rb, &one, (const cuDoubleComplex*)wC3[wi].p, rb,
                                 &zero, (const cuDoubleComplex*)wC3[wi].p, rb, (cuDoubleComplex*)Cc, m));
        TFMM_CUDA_CHECK(cudaGetLastError());
        TFMM_CUDA_CHECK(cudaStreamSynchronize(w.s));  // wC3 / wV are reused by this worker's next tensor
        ms_f[wi] += ms_since(tc);
        int* rk = &P.ranks[((size_t)T[t].g * 2 + T[t].alpha) * 3];
        rk[0] = rt; rk[1] = rp; rk[2] = rb;
    });
    const double wall = ms_since(t0);
    double sg = 0, se = 0, sf = 0;
    for (int i = 0; i < nw; ++i) { sg += ms_g[i]; se += ms_e[i]; sf += ms_f[i]; }
    const double tot = std::max(sg + se + sf, 1e-9);
    tm.gram3 += wall * sg / tot;
    tm.eig3 += wall * se / tot;
    tm.fac3 += wall * sf / tot;
}

}  // namespace

// Gauss-Legendre nodes and weights on [-1, 1], nodes ascending, by Newton's
// iteration on the three-term recurrence of P_n (Golub & Welsch give the same
// rule as eigenvalues of the Jacobi matrix).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int l = 2; l <= n; ++l) {
                const double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        // recompute the derivative at the converged node
        double p0 = 1.0, p1 = z;
        for (int l = 2; l <= n; ++l) {
            const double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
            p0 = p1;
            p1 = p2;
        }
        if (n == 1) { p1 = z; p0 = 1.0; }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    if (n % 2 == 1) x[n / 2] = 0.0;
}

void build_tucker_setup(Plan& P, const Mesh& M, cudaStream_t s) {
    (void)M;
    const auto t_all = std::chrono::steady_clock::now();
    const tfmm_params& prm = P.params;
    const int nd = P.n_dir;
    const bool keep_dense = prm.keep_dense != 0;
    TFMM_REQUIRE(prm.quad_order >= 1 && prm.quad_order <= kMaxQuad, "quad_order must be in 1..10");
    upload_quadrature(prm.quad_order, s);
    const int nq = prm.quad_order * prm.quad_order;

    // geometry and directions
    TFMM_CUDA_CHECK(device_malloc(&P.d_geom, sizeof(RwgGeom) * std::max<int64_t>(P.N, 1)));
    TFMM_CUDA_CHECK(cudaMemcpyAsync(P.d_geom, P.geom.data(), sizeof(RwgGeom) * P.N, cudaMemcpyHostToDevice, s));
    const std::vector<double> dirs = direction_table(P);
    DevBuf d_dirs(sizeof(double) * dirs.size());
    TFMM_CUDA_CHECK(cudaMemcpyAsync(d_dirs.p, dirs.data(), sizeof(double) * dirs.size(), cudaMemcpyHostToDevice, s));

    // dense FP32 copy
    if (keep_dense) {
        P.dense_elems = (int64_t)P.ld_dir * P.N * 2;
        TFMM_CUDA_CHECK(device_malloc(&P.d_dense, sizeof(float2) * std::max<int64_t>(P.dense_elems, 1)));
    }

    int nworkers = 8;
    if (const char* e = std::getenv("TFMM_SETUP_STREAMS")) nworkers = std::max(1, std::min(64, std::atoi(e)));
    std::vector<std::unique_ptr<Worker>> pool;
    for (int i = 0; i < nworkers; ++i) pool.emplace_back(new Worker());
    Timers timers;

    // batches of groups bounded by a device-memory budget
    size_t free_b = 0, total_b = 0;
    TFMM_CUDA_CHECK(cudaMemGetInfo(&free_b, &total_b));
    // tensors + projections + Grams, both alpha (an SVD plan keeps its projections whole)
    const double per_rwg = 16.0 * nd * 2 * (plan_is_svd(P) ? 4.5 : 3.2);
    const double budget = std::min<double>(0.35 * (double)free_b, 48e9);
    int64_t rwg_budget = (int64_t)std::max(1.0, budget / per_rwg);
    if (prm.batch_groups > 0) rwg_budget = INT64_MAX;

    P.f64.assign((size_t)P.G * 2, HostFactors64{});
    P.ranks.assign((size_t)P.G * 6, 0);
    double ms_ff = 0, ms_svd = 0;

    int g0 = 0;
    while (g0 < P.G) {
        int g1 = g0;
        int64_t rw = 0;
        while (g1 < P.G) {
            const int64_t nb = P.grp_off[g1 + 1] - P.grp_off[g1];
            if (g1 > g0 && (rw + nb > rwg_budget || (prm.batch_groups > 0 && g1 - g0 >= prm.batch_groups))) break;
            rw += nb;
            ++g1;
        }
        const int nbg = g1 - g0;
        // ---- far-fields of the batch
        auto t0 = std::chrono::steady_clock::now();
        std::vector<int64_t> rwg_off(nbg), out_off(nbg);
        std::vector<int> nbeta(nbg);
        std::vector<double> cen(3 * nbg);
        int64_t tot = 0;
        int maxnb = 0;
        for (int b = 0; b < nbg; ++b) {
            const int g = g0 + b;
            rwg_off[b] = P.grp_off[g];
            nbeta[b] = (int)(P.grp_off[g + 1] - P.grp_off[g]);
            maxnb = std::max(maxnb, nbeta[b]);
            out_off[b] = tot;
            tot += (int64_t)2 * nd * nbeta[b];
            for (int c = 0; c < 3; ++c) cen[3 * b + c] = P.centres[3 * g + c];
        }
        DevBuf d_A(sizeof(double2) * tot);
        DevBuf d_rwg_off(sizeof(int64_t) * nbg), d_out_off(sizeof(int64_t) * nbg), d_nb(sizeof(int) * nbg),
            d_cen(sizeof(double) * 3 * nbg);
        TFMM_CUDA_CHECK(cudaMemcpyAsync(d_rwg_off.p, rwg_off.data(), sizeof(int64_t) * nbg, cudaMemcpyHostToDevice, s));
        TFMM_CUDA_CHECK(cudaMemcpyAsync(d_out_off.p, out_off.data(), sizeof(int64_t) * nbg, cudaMemcpyHostToDevice, s));
        TFMM_CUDA_CHECK(cudaMemcpyAsync(d_nb.p, nbeta.data(), sizeof(int) * nbg, cudaMemcpyHostToDevice, s));
        TFMM_CUDA_CHECK(cudaMemcpyAsync(d_cen.p, cen.data(), sizeof(double) * 3 * nbg, cudaMemcpyHostToDevice, s));
        FFArgs fa;
        fa.geom = P.d_geom;
        fa.grp_rwg = P.d_grp_rwg;
        fa.rwg_off = d_rwg_off.as<int64_t>();
        fa.out_off = d_out_off.as<int64_t>();
        fa.nbeta = d_nb.as<int>();
        fa.centre = d_cen.as<double>();
        fa.dirs = d_dirs.as<double>();
        fa.out = d_A.as<double2>();
        fa.k = P.k;
        fa.n_dir = nd;
        fa.nq = nq;
        dim3 grid((nd + kFFThreads - 1) / kFFThreads, (maxnb + kFFRwgs - 1) / kFFRwgs, nbg);
        farfield_kernel<<<grid, kFFThreads, 0, s>>>(fa);
        TFMM_CUDA_CHECK(cudaGetLastError());
        if (keep_dense) {
            for (int b = 0; b < nbg; ++b)
                for (int al = 0; al < 2; ++al) {
                    const int64_t dst = ((int64_t)2 * P.grp_off[g0 + b] + (int64_t)al * nbeta[b]) * P.ld_dir;
                    to_f32_kernel<<<grid1d((int64_t)nd * nbeta[b]), 256, 0, s>>>(
                        d_A.as<double2>() + out_off[b] + (int64_t)al * nd * nbeta[b], nd, nbeta[b], nd,
                        P.d_dense + dst, P.ld_dir);
                }
            TFMM_CUDA_CHECK(cudaGetLastError());
        }
        TFMM_CUDA_CHECK(cudaStreamSynchronize(s));
        ms_ff += ms_since(t0);

        // ---- HOSVD of the batch
        t0 = std::chrono::steady_clock::now();
        std::vector<Tensor> T;
        for (int b = 0; b < nbg; ++b)
            for (int al = 0; al < 2; ++al)
                T.push_back(Tensor{g0 + b, al, nbeta[b], d_A.as<double2>() + out_off[b] + (int64_t)al * nd * nbeta[b]});
        hosvd_batch(P, T, pool, s, timers);
        ms_svd += ms_since(t0);
        g0 = g1;
    }
    const auto t0 = std::chrono::steady_clock::now();
    pack_factors_fp32(P, s);
    TFMM_CUDA_CHECK(cudaStreamSynchronize(s));
    P.setup_ms[0] = ms_ff;
    P.setup_ms[1] = ms_svd;
    P.setup_ms[2] = ms_since(t0);
    P.setup_ms[3] = ms_since(t_all);
    if (std::getenv("TFMM_VERBOSE"))
        std::fprintf(stderr,
                     "[tfmm setup] far-field %.1f ms, HOSVD %.1f ms (mode1 %.1f, mode2 %.1f, mode3 gram %.1f, "
                     "mode3 eig %.1f, mode3 factors %.1f), pack %.1f ms, %d workers\n",
                     ms_ff, ms_svd, timers.mode1, timers.mode2, timers.gram3, timers.eig3, timers.fac3,
                     P.setup_ms[2], (int)pool.size());
}

void farfield_group_host(const Plan& P, int g, double2* At, double2* Ap, cudaStream_t s) {
    TFMM_REQUIRE(P.has_geometry && P.d_geom, "plan has no geometry (built from factors)");
    TFMM_REQUIRE(g >= 0 && g < P.G, "group index out of range");
    upload_quadrature(P.params.quad_order, s);
    const int nb = (int)(P.grp_off[g + 1] - P.grp_off[g]);
    const int nd = P.n_dir;
    const std::vector<double> dirs = direction_table(P);
    DevBuf d_dirs(sizeof(double) * dirs.size()), d_A(sizeof(double2) * 2 * (int64_t)nd * nb);
    DevBuf d_rwg_off(sizeof(int64_t)), d_out_off(sizeof(int64_t)), d_nb(sizeof(int)), d_cen(sizeof(double) * 3);
    const int64_t ro = P.grp_off[g], oo = 0;
    TFMM_CUDA_CHECK(cudaMemcpyAsync(d_dirs.p, dirs.data(), sizeof(double) * dirs.size(), cudaMemcpyHostToDevice, s));
    TFMM_CUDA_CHECK(cudaMemcpyAsync(d_rwg_off.p, &ro, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    TFMM_CUDA_CHECK(cudaMemcpyAsync(d_out_off.p, &oo, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    TFMM_CUDA_CHECK(cudaMemcpyAsync(d_nb.p, &nb, sizeof(int), cudaMemcpyHostToDevice, s));
    TFMM_CUDA_CHECK(cudaMemcpyAsync(d_cen.p, &P.centres[3 * g], sizeof(double) * 3, cudaMemcpyHostToDevice, s));
    FFArgs fa;
    fa.geom = P.d_geom;
    fa.grp_rwg = P.d_grp_rwg;
    fa.rwg_off = d_rwg_off.as<int64_t>();
    fa.out_off = d_out_off.as<int64_t>();
    fa.nbeta = d_nb.as<int>();
    fa.centre = d_cen.as<double>();
    fa.dirs = d_dirs.as<double>();
    fa.out = d_A.as<double2>();
    fa.k = P.k;
    fa.n_dir = nd;
    fa.nq = P.params.quad_order * P.params.quad_order;
    dim3 grid((nd + kFFThreads - 1) / kFFThreads, (nb + kFFRwgs - 1) / kFFRwgs, 1);
    farfield_kernel<<<grid, kFFThreads, 0, s>>>(fa);
    TFMM_CUDA_CHECK(cudaGetLastError());
    TFMM_CUDA_CHECK(cudaMemcpyAsync(At, d_A.p, sizeof(double2) * (int64_t)nd * nb, cudaMemcpyDeviceToHost, s));
    TFMM_CUDA_CHECK(cudaMemcpyAsync(Ap, d_A.as<double2>() + (int64_t)nd * nb, sizeof(double2) * (int64_t)nd * nb,
                                    cudaMemcpyDeviceToHost, s));
    TFMM_CUDA_CHECK(cudaStreamSynchronize(s));
}

void planewave_rhs(const Plan& P, const double* khat, const double* pol, int R, float2* V, cudaStream_t s) {
    TFMM_REQUIRE(P.has_geometry && P.d_geom, "plan has no geometry (built from factors)");
    upload_quadrature(P.params.quad_order, s);
    DevBuf d_k(sizeof(double) * 3 * R), d_p(sizeof(double) * 3 * R);
    TFMM_CUDA_CHECK(cudaMemcpyAsync(d_k.p, khat, sizeof(double) * 3 * R, cudaMemcpyHostToDevice, s));
    TFMM_CUDA_CHECK(cudaMemcpyAsync(d_p.p, pol, sizeof(double) * 3 * R, cudaMemcpyHostToDevice, s));
    PWArgs a;
    a.geom = P.d_geom;
    a.khat = d_k.as<double>();
    a.pol = d_p.as<double>();
    a.V = V;
    a.k = P.k;
    a.n = P.N;
    a.R = R;
    a.nq = P.params.quad_order * P.params.quad_order;
    dim3 grid((unsigned)((P.N + 255) / 256), R);
    planewave_kernel<<<grid, 256, 0, s>>>(a);
    TFMM_CUDA_CHECK(cudaGetLastError());
    TFMM_CUDA_CHECK(cudaStreamSynchronize(s));
}

// ------------------------------------------------ allocation-free excitation
// Some callers cannot allocate device memory while they call into the library:
// applications whose device memory is all handed out by their own pool
// allocator (a library cudaMalloc would fail or fragment that pool), and loops
// that cannot afford the device-wide synchronisation a cudaFree implies.  For
// them tfmm_planewave_noalloc stages the incidence table in this fixed array
// instead of a per-call allocation.  It holds kNoAllocMaxIncidences directions
// and polarisations (6 doubles each, 48 KiB); every GPU that loads the library
// keeps it until the process exits.  All calls share it.
constexpr int kNoAllocMaxIncidences = 1024;
static __device__ __align__(256) double g_pw_table[6 * kNoAllocMaxIncidences];

namespace {
std::mutex g_pw_table_mu;
double* g_pw_table_addr[256] = {};
// Host staging copy of the incidence table.  The caller's khat / pol may be
// pinned, in which case a copy straight from them could still be in flight
// when the call returns; this array is ordinary pageable memory, which
// cudaMemcpyAsync has consumed (copied to its own staging area) by the time it
// returns, so the caller may reuse its arrays at once.  Guarded by
// g_pw_stage_mu for the duration of the two copies.
std::mutex g_pw_stage_mu;
double g_pw_stage[6 * kNoAllocMaxIncidences];

// Device address of g_pw_table on the current device, looked up once per device
// (a host-side reference to g_pw_table is only a stand-in, not that address).
double* pw_table_address() {
    int dev = 0;
    TFMM_CUDA_CHECK(cudaGetDevice(&dev));
    TFMM_REQUIRE(dev >= 0 && dev < 256, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_pw_table_mu);
    if (!g_pw_table_addr[dev]) {
        void* p = nullptr;
        TFMM_CUDA_CHECK(cudaGetSymbolAddress(&p, g_pw_table));
        g_pw_table_addr[dev] = static_cast<double*>(p);
    }
    return g_pw_table_addr[dev];
}
}  // namespace

void planewave_rhs_noalloc(const Plan& P, const double* khat, const double* pol, int R, float2* V, cudaStream_t s) {
    TFMM_REQUIRE(P.has_geometry && P.d_geom, "plan has no geometry (built from factors)");
    TFMM_REQUIRE(R >= 1 && R <= kNoAllocMaxIncidences,
                 "R = " + std::to_string(R) + " incidences exceed the static table of " +
                     std::to_string(kNoAllocMaxIncidences) + "; split the sweep or call tfmm_planewave");
    double* table = pw_table_address();
    upload_quadrature(P.params.quad_order, s);
    // every entry the kernel reads is overwritten here: nothing has to start at zero
    {
        std::lock_guard<std::mutex> lock(g_pw_stage_mu);
        std::memcpy(g_pw_stage, khat, sizeof(double) * 3 * R);
        std::memcpy(g_pw_stage + 3 * kNoAllocMaxIncidences, pol, sizeof(double) * 3 * R);
        TFMM_CUDA_CHECK(cudaMemcpyAsync(table, g_pw_stage, sizeof(double) * 3 * R, cudaMemcpyHostToDevice, s));
        TFMM_CUDA_CHECK(cudaMemcpyAsync(table + 3 * kNoAllocMaxIncidences, g_pw_stage + 3 * kNoAllocMaxIncidences,
                                        sizeof(double) * 3 * R, cudaMemcpyHostToDevice, s));
    }
    PWArgs a;
    a.geom = P.d_geom;
    a.khat = table;
    a.pol = table + 3 * kNoAllocMaxIncidences;
    a.V = V;
    a.k = P.k;
    a.n = P.N;
    a.R = R;
    a.nq = P.params.quad_order * P.params.quad_order;
    dim3 grid((unsigned)((P.N + 255) / 256), R);
    planewave_kernel<<<grid, 256, 0, s>>>(a);
    TFMM_CUDA_CHECK(cudaGetLastError());
}

}  // namespace tfmm
