// Synthetic observations from the generative signal model (eq. observation-
// generative, Sec. II-B): z = sum_k rho_k psi(p, p_sfv,k) + n, FP64 signal,
// noise CN(0, eta I) with eta from the sum-channel SNR of the first step
// (Sec. V-A).  Test and benchmark harness; not part of the filter step.
#include "bp_internal.cuh"
#include "bp_kernels.cuh"

namespace bp {

__device__ inline double2 steer_elem(const DevGeom& G, int j, int k, const double* p, const double* sfv, bool los) {
    const PathGeo pg = path_geo(G, j, p[0], p[1], p[2], sfv[0], sfv[1], sfv[2], los);
    const int Nm = G.My * G.Mz;
    const int f = k / Nm, ym = k - f * Nm, y = ym / G.Mz, m = ym - y * G.Mz;
    const double A = G.lam / (4.0 * M_PI * pg.d);
    // phase in cycles: -(fc + f) d/c + (p_y u_y + p_z u_z)/lambda
    const double cyc = -frac_c(pg.d / G.lam) - frac_c(G.f[f] * pg.d / G.c) + (G.py[y] * pg.uy + G.pz[m] * pg.uz) / G.lam;
    double s, c;
    sincospi(2.0 * frac_c(cyc), &s, &c);
    return make_double2(A * c, A * s);
}

__global__ void k_synth_clean(DevGeom G, int n_steps, const double* x_pos, int K, const double* sfv,
                              const double* rho, const int* c_off, const double* c_sfv, const double* c_rho,
                              double* zbuf) {
    const int J = G.J, Nz = G.Nz;
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)n_steps * J * Nz) return;
    const int k = (int)(idx % Nz);
    const int j = (int)((idx / Nz) % J);
    const int t = (int)(idx / ((long)Nz * J));
    const double* p = x_pos + 3 * t;
    double2 acc = make_double2(0.0, 0.0);
    const double zero[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c <= K; ++c) {
        const double* r = rho + 2 * (((size_t)t * J + j) * (K + 1) + c);
        if (r[0] == 0.0 && r[1] == 0.0) continue;
        const double2 ps = steer_elem(G, j, k, p, c == 0 ? zero : sfv + 3 * (c - 1), c == 0);
        const double2 u = zmul(make_double2(r[0], r[1]), ps);
        acc.x += u.x; acc.y += u.y;
    }
    for (int c = c_off[t]; c < c_off[t + 1]; ++c) {
        const double* r = c_rho + 2 * ((size_t)c * J + j);
        const double2 ps = steer_elem(G, j, k, p, c_sfv + 3 * c, false);
        const double2 u = zmul(make_double2(r[0], r[1]), ps);
        acc.x += u.x; acc.y += u.y;
    }
    reinterpret_cast<double2*>(zbuf)[idx] = acc;
}

// sum-channel power of the first step without clutter: launched on a clean
// buffer that holds only the true components
__global__ void k_power(DevGeom G, const double* zbuf, double* out) {
    const int n = G.J * G.Nz;
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double2 v = reinterpret_cast<const double2*>(zbuf)[i];
        acc += v.x * v.x + v.y * v.y;
    }
    __shared__ double red[32];
    acc = warp_sum_d(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        *out = s / n;
    }
}

__global__ void k_synth_noise(DevGeom G, int n_steps, int step0, const double* zbuf, double eta, uint32_t k0,
                              uint32_t k1, float* z_out) {
    const int J = G.J, Nz = G.Nz;
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)n_steps * J * Nz) return;
    const int k = (int)(idx % Nz);
    const int j = (int)((idx / Nz) % J);
    const int t = (int)(idx / ((long)Nz * J));
    const U4 r = philox((uint32_t)k, (uint32_t)(step0 + t), (RNG_SYNTH_NOISE << 16) | (uint32_t)j, 0u, k0, k1);
    const double rad = sqrt(-2.0 * log(u32d(r.x)));
    double s, c;
    sincospi(2.0 * u32d(r.y), &s, &c);
    const double sd = sqrt(eta / 2.0);
    const double2 v = reinterpret_cast<const double2*>(zbuf)[idx];
    z_out[2 * idx] = (float)(v.x + sd * rad * c);
    z_out[2 * idx + 1] = (float)(v.y + sd * rad * s);
}

void launch_synth(const DevGeom& G, int n_steps, int step0, const double* x_pos, int K, const double* sfv,
                  const double* rho, const int* c_off, const double* c_sfv, const double* c_rho,
                  double* zbuf, uint32_t, uint32_t, cudaStream_t st) {
    (void)step0;
    const long n = (long)n_steps * G.J * G.Nz;
    k_synth_clean<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(G, n_steps, x_pos, K, sfv, rho, c_off, c_sfv, c_rho, zbuf);
}

void launch_power(const DevGeom& G, const double* zbuf, double* out, cudaStream_t st) {
    k_power<<<1, 512, 0, st>>>(G, zbuf, out);
}

void launch_synth_noise(const DevGeom& G, int n_steps, int step0, const double* zbuf, double eta, uint32_t k0,
                        uint32_t k1, float* z_out, cudaStream_t st) {
    const long n = (long)n_steps * G.J * G.Nz;
    k_synth_noise<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(G, n_steps, step0, zbuf, eta, k0, k1, z_out);
}

}  // namespace bp
