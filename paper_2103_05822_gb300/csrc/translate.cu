// Translation stage of the FMM-FFT (Sec. II.A, between Eqs. 3 and 5; refs. [7, 8]),
// with the translation operator of the addition theorem (ref. [25]):
//
//   g_v(k_i) = c sum_{v' far from v} T_L(k_i, r_v - r_v') F_v'(k_i),
//   T_L(k, X) = sum_{l=0}^{L} (-j)^l (2l + 1) h_l^(2)(k |X|) P_l(k . X / |X|),
//   c = -j k / (16 pi^2),
//
// for every box v, direction i and component alpha; boxes are far when their grid
// indices differ by 2 or more in some coordinate (touching boxes belong to the near
// field).  T depends on the boxes only through their index difference, so for each
// direction the sum is a discrete 3-D convolution over the box grid: the spectra are
// scattered into a zero-padded grid of N_x x N_y x N_z >= (2K - 1)^3 points,
// transformed, multiplied by the transform of c T (built once, FP64, then stored
// FP32) and transformed back; the FFTs are cuFFT's, everything else is kernels here.
//
// Layout: the 2 N_dir transforms of one right-hand side one after the other, transform
// j = alpha N_dir + i holding grid point s at j N_grid + s (each transform contiguous,
// the layout batched FFTs run fastest in); the kernel's transform likewise, N_dir x N_grid.
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace tfmm {

namespace {

#define CUFFT_CHECK(call)                                                                           \
    do {                                                                                            \
        cufftResult r_ = (call);                                                                    \
        if (r_ != CUFFT_SUCCESS)                                                                    \
            fail(r_ == CUFFT_ALLOC_FAILED ? TFMM_OOM : TFMM_CUDA,                                    \
                 std::string(#call) + " failed with cuFFT status " + std::to_string((int)r_));     \
    } while (0)

constexpr int kMaxL = 512;

// c T_L(k_i, X(s)) for the grid point s (signed index differences d, far ones only), FP64:
// h_l^(2)(k|X|) by the upward three-term recurrence of the spherical Bessel functions
// (stable for h^(2) = j - i y, whose magnitude grows with l), P_l(cos) by Bonnet's recurrence.
__global__ void translation_kernel(const double* __restrict__ khat, int n_dir, int L, double k, double a, int Nx,
                                   int Ny, int Nz, int Kx, int Ky, int Kz, int64_t Ns, double2* __restrict__ T) {
    __shared__ double2 h[kMaxL + 1];
    __shared__ double xh[3];
    __shared__ int far;
    const int64_t s = blockIdx.x;
    const int sx = (int)(s % Nx), sy = (int)((s / Nx) % Ny), sz = (int)(s / ((int64_t)Nx * Ny));
    const int dx = sx < Nx - sx ? sx : sx - Nx, dy = sy < Ny - sy ? sy : sy - Ny, dz = sz < Nz - sz ? sz : sz - Nz;
    if (threadIdx.x == 0) {
        const int m = max(abs(dx), max(abs(dy), abs(dz)));
        far = (m >= 2 && abs(dx) < Kx && abs(dy) < Ky && abs(dz) < Kz) ? 1 : 0;
        if (far) {
            const double X[3] = {dx * a, dy * a, dz * a};
            const double r = sqrt(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
            for (int c = 0; c < 3; ++c) xh[c] = X[c] / r;
            const double x = k * r, sn = sin(x), cs = cos(x);
            // h_0 = j_0 - i y_0, h_1 = j_1 - i y_1
            h[0] = make_double2(sn / x, cs / x);
            if (L >= 1) h[1] = make_double2(sn / (x * x) - cs / x, cs / (x * x) + sn / x);
            for (int l = 1; l < L; ++l) {
                const double f = (2.0 * l + 1.0) / x;
                h[l + 1] = make_double2(f * h[l].x - h[l - 1].x, f * h[l].y - h[l - 1].y);
            }
        }
    }
    __syncthreads();
    const double2 c = make_double2(0.0, -k / (16.0 * 3.14159265358979323846 * 3.14159265358979323846));
    for (int i = threadIdx.x; i < n_dir; i += blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        if (far) {
            const double ct = khat[3 * i] * xh[0] + khat[3 * i + 1] * xh[1] + khat[3 * i + 2] * xh[2];
            double pm = 0.0, p = 1.0;  // P_{l-1}, P_l
            for (int l = 0; l <= L; ++l) {
                if (l == 1) {
                    pm = 1.0;
                    p = ct;
                } else if (l >= 2) {
                    const double pn = ((2.0 * l - 1.0) * ct * p - (l - 1.0) * pm) / l;
                    pm = p;
                    p = pn;
                }
                // (-j)^l (2l + 1) P_l h_l
                const double w = (2.0 * l + 1.0) * p;
                double2 t = make_double2(w * h[l].x, w * h[l].y);
                switch (l & 3) {
                    case 1: t = make_double2(t.y, -t.x); break;   // * (-j)
                    case 2: t = make_double2(-t.x, -t.y); break;  // * (-1)
                    case 3: t = make_double2(-t.y, t.x); break;   // * (+j)
                    default: break;
                }
                acc.x += t.x;
                acc.y += t.y;
            }
            acc = make_double2(c.x * acc.x - c.y * acc.y, c.x * acc.y + c.y * acc.x);
        }
        T[(int64_t)i * Ns + s] = acc;
    }
}

__global__ void to_f32_kernel(const double2* __restrict__ in, int64_t n, float2* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = make_float2((float)in[e].x, (float)in[e].y);
}

// grid[j][cell(g)] = spectra[g][j] for every group g and j < 2 N_dir (the rest of the
// grid was zeroed)
__global__ void scatter_kernel(const float2* __restrict__ spec, const int* __restrict__ group_cell, int G, int nb,
                               int64_t Ns, float2* __restrict__ grid) {
    const int64_t total = (int64_t)G * nb;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int g = (int)(e / nb), j = (int)(e - (int64_t)g * nb);
        grid[(int64_t)j * Ns + group_cell[g]] = spec[e];
    }
}

// grid[alpha N_dir + i][s] *= That[i][s]
__global__ void multiply_kernel(float2* __restrict__ grid, const float2* __restrict__ That, int64_t Ns, int n_dir) {
    const int64_t per = (int64_t)n_dir * Ns, total = 2 * per;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const float2 t = That[e < per ? e : e - per], v = grid[e];
        grid[e] = make_float2(v.x * t.x - v.y * t.y, v.x * t.y + v.y * t.x);
    }
}

// spectra_in[g][j] = grid[j][cell(g)] / Ns (the inverse transform is unnormalised)
__global__ void gather_kernel(const float2* __restrict__ grid, const int* __restrict__ group_cell, int G, int nb,
                              int64_t Ns, float scale, float2* __restrict__ spec) {
    const int64_t total = (int64_t)G * nb;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int g = (int)(e / nb), j = (int)(e - (int64_t)g * nb);
        const float2 v = grid[(int64_t)j * Ns + group_cell[g]];
        spec[e] = make_float2(scale * v.x, scale * v.y);
    }
}

int grid_blocks(int64_t total) { return (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 64)); }

// smallest n >= m whose prime factors are 2, 3, 5 or 7 (fast cuFFT sizes)
int fft_size(int m) {
    for (int n = std::max(m, 1);; ++n) {
        int v = n;
        for (int p : {2, 3, 5, 7})
            while (v % p == 0) v /= p;
        if (v == 1) return n;
    }
}

}  // namespace

TransPlan::~TransPlan() {
    if (fft) cufftDestroy((cufftHandle)fft);
}

void build_translation(Plan& P, cudaStream_t s) {
    if (P.trans) return;
    TFMM_REQUIRE(P.has_geometry && !P.centres.empty(), "translation needs box centres: a plan made by tfmm_plan_create");
    TFMM_REQUIRE(P.L <= kMaxL, "bandwidth L too large for the translation kernel");
    auto T = std::make_unique<TransPlan>();
    const double a = P.params.box;
    // integer box coordinates relative to the lowest centre (differences are what matter)
    double lo[3] = {INFINITY, INFINITY, INFINITY};
    for (int g = 0; g < P.G; ++g)
        for (int c = 0; c < 3; ++c) lo[c] = std::min(lo[c], P.centres[3 * (size_t)g + c]);
    std::vector<int> bi((size_t)P.G * 3);
    int K[3] = {1, 1, 1};
    for (int g = 0; g < P.G; ++g)
        for (int c = 0; c < 3; ++c) {
            const int v = (int)std::lround((P.centres[3 * (size_t)g + c] - lo[c]) / a);
            bi[3 * (size_t)g + c] = v;
            K[c] = std::max(K[c], v + 1);
        }
    for (int c = 0; c < 3; ++c) T->N[c] = fft_size(2 * K[c] - 1);
    T->Ns = (int64_t)T->N[0] * T->N[1] * T->N[2];
    const int nd = P.n_dir;
    T->nb = 2 * nd;
    std::vector<int> group_cell(P.G);
    for (int g = 0; g < P.G; ++g) {
        const int64_t cell = bi[3 * (size_t)g] + (int64_t)T->N[0] * (bi[3 * (size_t)g + 1] + (int64_t)T->N[1] * bi[3 * (size_t)g + 2]);
        group_cell[g] = (int)cell;
    }
    TFMM_CUDA_CHECK(device_malloc(&T->group_cell.p, sizeof(int) * std::max(P.G, 1)));
    TFMM_CUDA_CHECK(cudaMemcpy(T->group_cell.p, group_cell.data(), sizeof(int) * P.G, cudaMemcpyHostToDevice));
    // directions k_i
    std::vector<double> kh((size_t)nd * 3);
    for (int ip = 0; ip < P.n_phi; ++ip)
        for (int it = 0; it < P.n_theta; ++it) {
            const double t = P.theta[it], ph = P.phi[ip];
            double* d = &kh[3 * ((size_t)it + (size_t)P.n_theta * ip)];
            d[0] = std::sin(t) * std::cos(ph);
            d[1] = std::sin(t) * std::sin(ph);
            d[2] = std::cos(t);
        }
    {
        DeviceBuffer d_kh, d_T;
        TFMM_CUDA_CHECK(device_malloc(&d_kh.p, sizeof(double) * kh.size()));
        TFMM_CUDA_CHECK(cudaMemcpy(d_kh.p, kh.data(), sizeof(double) * kh.size(), cudaMemcpyHostToDevice));
        TFMM_CUDA_CHECK(device_malloc(&d_T.p, sizeof(double2) * T->Ns * nd));
        translation_kernel<<<(unsigned)T->Ns, 128, 0, s>>>(static_cast<const double*>(d_kh.p), nd, P.L, P.k, a,
                                                           T->N[0], T->N[1], T->N[2], K[0], K[1], K[2], T->Ns,
                                                           static_cast<double2*>(d_T.p));
        TFMM_CUDA_CHECK(cudaGetLastError());
        // forward transform of every direction's kernel over the grid (FP64), then FP32
        int n[3] = {T->N[2], T->N[1], T->N[0]};
        cufftHandle h64 = 0;
        CUFFT_CHECK(cufftPlanMany(&h64, 3, n, n, 1, (int)T->Ns, n, 1, (int)T->Ns, CUFFT_Z2Z, nd));
        cufftSetStream(h64, s);
        const cufftResult r64 = cufftExecZ2Z(h64, static_cast<cufftDoubleComplex*>(d_T.p),
                                             static_cast<cufftDoubleComplex*>(d_T.p), CUFFT_FORWARD);
        cufftDestroy(h64);
        CUFFT_CHECK(r64);
        TFMM_CUDA_CHECK(device_malloc(&T->That.p, sizeof(float2) * T->Ns * nd));
        to_f32_kernel<<<grid_blocks(T->Ns * nd), 256, 0, s>>>(static_cast<const double2*>(d_T.p), T->Ns * nd,
                                                              static_cast<float2*>(T->That.p));
        TFMM_CUDA_CHECK(cudaGetLastError());
        TFMM_CUDA_CHECK(cudaStreamSynchronize(s));
    }
    TFMM_CUDA_CHECK(device_malloc(&T->grid.p, sizeof(float2) * T->Ns * T->nb));
    int n[3] = {T->N[2], T->N[1], T->N[0]};
    cufftHandle h = 0;
    CUFFT_CHECK(cufftPlanMany(&h, 3, n, n, 1, (int)T->Ns, n, 1, (int)T->Ns, CUFFT_C2C, T->nb));
    T->fft = (int)h;
    P.trans = std::move(T);
}

void launch_translate(Plan& P, const float2* spec_out, int R, float2* spec_in, cudaStream_t s) {
    build_translation(P, s);
    TransPlan& T = *P.trans;
    float2* grid = static_cast<float2*>(T.grid.p);
    CUFFT_CHECK(cufftSetStream((cufftHandle)T.fft, s));
    for (int r = 0; r < R; ++r) {
        const int64_t off = (int64_t)r * P.G * T.nb;
        TFMM_CUDA_CHECK(cudaMemsetAsync(grid, 0, sizeof(float2) * T.Ns * T.nb, s));
        scatter_kernel<<<grid_blocks((int64_t)P.G * T.nb), 256, 0, s>>>(
            spec_out + off, static_cast<const int*>(T.group_cell.p), P.G, T.nb, T.Ns, grid);
        TFMM_CUDA_CHECK(cudaGetLastError());
        CUFFT_CHECK(cufftExecC2C((cufftHandle)T.fft, reinterpret_cast<cufftComplex*>(grid),
                                 reinterpret_cast<cufftComplex*>(grid), CUFFT_FORWARD));
        multiply_kernel<<<grid_blocks(T.Ns * T.nb), 256, 0, s>>>(grid, static_cast<const float2*>(T.That.p), T.Ns,
                                                                 P.n_dir);
        TFMM_CUDA_CHECK(cudaGetLastError());
        CUFFT_CHECK(cufftExecC2C((cufftHandle)T.fft, reinterpret_cast<cufftComplex*>(grid),
                                 reinterpret_cast<cufftComplex*>(grid), CUFFT_INVERSE));
        gather_kernel<<<grid_blocks((int64_t)P.G * T.nb), 256, 0, s>>>(
            grid, static_cast<const int*>(T.group_cell.p), P.G, T.nb, T.Ns, 1.0f / (float)T.Ns, spec_in + off);
        TFMM_CUDA_CHECK(cudaGetLastError());
    }
}

}  // namespace tfmm
