// Posterior Cramer-Rao lower bounds (Sec. VI; Supplementary Sec. S-VII), FP64.
//
// k_pcrlb_fim: one block per state realisation m; per PA j the block forms the local
// channel FIM J_ch = (2/eta) Re(D^H D) (Table S-I; D = d mu / d [elevations, azimuths,
// delays, phases, moduli], built in chunks of elements in shared memory) and adds
// G_j J_ch G_j^T to the realisation's FIM, G_j the Jacobian from local channel parameters
// to the global ones (Sec. S-VII-B; the SFV block is the full derivative of the
// PA-to-virtual-MT vector).  Each thread owns fixed entries of the FIM, so the sums run in
// a fixed order.  k_pcrlb_mean averages the realisations (the Bayesian snapshot FIM).
// k_pcrlb_recursion: one block runs J_{n|n} = J_B,n + (F J_{n-1|n-1}^-1 F^T + Q)^-1 with
// Cholesky inversions and writes PEB and MEB per step.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "bp_handle.cuh"

namespace bp {

constexpr int PCRLB_KMAX = 15;      // surfaces (components K~ = K + 1 <= 16)
constexpr int PCRLB_CH = 32;        // elements per chunk of D

struct PcrlbDims {
    int K, Kt, J, nph, o_sfv, o_ph, o_a, o_eta, dim, L;   // L = 5 K~ + 1 local parameters
    __host__ __device__ PcrlbDims(int K_, int J_, bool coherent)
        : K(K_), Kt(K_ + 1), J(J_), nph(coherent ? K_ + 1 : (K_ + 1) * J_), o_sfv(6), o_ph(6 + 3 * K_),
          o_a(6 + 3 * K_ + (coherent ? K_ + 1 : (K_ + 1) * J_)),
          o_eta(6 + 3 * K_ + (coherent ? K_ + 1 : (K_ + 1) * J_) + (K_ + 1) * J_),
          dim(6 + 3 * K_ + (coherent ? K_ + 1 : (K_ + 1) * J_) + (K_ + 1) * J_ + 1), L(5 * (K_ + 1) + 1) {}
};

__device__ inline double2 cisd(double cycles) {
    const double f = cycles - rint(cycles);
    double s, c;
    sincospi(2.0 * f, &s, &c);
    return make_double2(c, s);
}

// local vector r' = R^T H (p - p_va) of component k (k = 0: LoS) at PA j, and H
__device__ inline void comp_geometry(const DevGeom& G, int j, const double* p, const double* s, bool los,
                                     double rp[3], double H[9]) {
    double r[3];
    if (los) {
        for (int i = 0; i < 3; ++i) r[i] = p[i] - G.p_pa[j][i];
        for (int i = 0; i < 9; ++i) H[i] = (i % 4 == 0) ? 1.0 : 0.0;
    } else {
        const double n2 = s[0] * s[0] + s[1] * s[1] + s[2] * s[2];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) H[3 * a + b] = (a == b ? 1.0 : 0.0) - 2.0 * s[a] * s[b] / n2;
        // r_breve = H p + s - p_pa (the virtual MT seen from the PA)
        for (int a = 0; a < 3; ++a) r[a] = H[3 * a] * p[0] + H[3 * a + 1] * p[1] + H[3 * a + 2] * p[2] + s[a] - G.p_pa[j][a];
    }
    const double* R = G.R[j];
    for (int c = 0; c < 3; ++c) rp[c] = R[c] * r[0] + R[3 + c] * r[1] + R[6 + c] * r[2];
}

// rows of G_j touched by local parameter u (at most 7: MT position, SFV k, phase / modulus / eta)
struct GCol { int n; int row[7]; double w[7]; };

__global__ void __launch_bounds__(256) k_pcrlb_fim(DevGeom G, int K, int coherent, const double* __restrict__ xs,
                                                   const double* __restrict__ sfvs, const double* __restrict__ rhos,
                                                   double eta, double* __restrict__ fims) {
    extern __shared__ double2 smp[];
    const PcrlbDims dd(K, G.J, coherent != 0);
    const int Kt = dd.Kt, L = dd.L, Lg = 5 * Kt, Nz = G.Nz, Nm = G.My * G.Mz;
    const int m = blockIdx.x, tid = threadIdx.x;
    double2* Dc = smp;                                            // [PCRLB_CH][5 K~]
    double* Jch = reinterpret_cast<double*>(Dc + PCRLB_CH * Lg);  // [L][L]
    GCol* gc = reinterpret_cast<GCol*>(Jch + L * L);              // [L]
    double* geo = reinterpret_cast<double*>(gc + L);              // [K~][8]: tau, theta, az per component
    double* lw = geo + 8 * Kt;                                    // [7 L] G's nonzeros by row: weights
    int* lu = reinterpret_cast<int*>(lw + 7 * L);                 // [7 L] their local index
    int* roff = lu + 7 * L;                                       // [dim + 1] row offsets
    const double* x = xs + (size_t)m * 6;
    const double* sv = sfvs + (size_t)m * K * 3;
    double* fim = fims + (size_t)m * dd.dim * dd.dim;
    for (int t = tid; t < dd.dim * dd.dim; t += blockDim.x) fim[t] = 0.0;
    for (int t = tid; t < 7 * L; t += blockDim.x) lu[t] = -1;
    const double lam = G.lam;
    for (int j = 0; j < G.J; ++j) {
        const double* rho = rhos + ((size_t)m * G.J + j) * Kt * 2;
        __syncthreads();
        // per component: spherical coordinates and the Jacobian columns (thread k)
        for (int k = tid; k < Kt; k += blockDim.x) {
            double rp[3], H[9];
            comp_geometry(G, j, x, k > 0 ? sv + 3 * (k - 1) : nullptr, k == 0, rp, H);
            const double d = sqrt(rp[0] * rp[0] + rp[1] * rp[1] + rp[2] * rp[2]);
            const double n2 = rp[0] * rp[0] + rp[1] * rp[1];
            geo[8 * k + 0] = d / G.c;
            geo[8 * k + 1] = acos(rp[2] / d);
            geo[8 * k + 2] = atan2(rp[1], rp[0]);
            // d(theta, az, tau, carrier phase) / d r'
            double ds[4][3];
            const double nn = sqrt(n2);
            for (int c = 0; c < 3; ++c) {
                ds[0][c] = (c < 2 ? rp[c] * rp[2] : -n2) / (d * d * nn);
                ds[1][c] = (c == 0 ? -rp[1] : (c == 1 ? rp[0] : 0.0)) / n2;
                ds[2][c] = rp[c] / (G.c * d);
                ds[3][c] = -2.0 * M_PI * rp[c] / (lam * d);
            }
            const double* R = G.R[j];
            double B[9];   // SFV block: I - 2 p s^T / |s|^2 - 2 (p . s) / |s|^2 H
            if (k > 0) {
                const double* s = sv + 3 * (k - 1);
                const double sn2 = s[0] * s[0] + s[1] * s[1] + s[2] * s[2];
                const double ps = x[0] * s[0] + x[1] * s[1] + x[2] * s[2];
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        B[3 * a + b] = (a == b ? 1.0 : 0.0) - 2.0 * x[a] * s[b] / sn2 - 2.0 * ps / sn2 * H[3 * a + b];
            }
            for (int q = 0; q < 4; ++q) {
                double Rd[3];   // R ds
                for (int a = 0; a < 3; ++a) Rd[a] = R[3 * a] * ds[q][0] + R[3 * a + 1] * ds[q][1] + R[3 * a + 2] * ds[q][2];
                GCol col;
                col.n = 0;
                for (int a = 0; a < 3; ++a) {
                    col.row[col.n] = a;
                    col.w[col.n++] = H[3 * a] * Rd[0] + H[3 * a + 1] * Rd[1] + H[3 * a + 2] * Rd[2];
                }
                if (k > 0)
                    for (int a = 0; a < 3; ++a) {
                        col.row[col.n] = dd.o_sfv + 3 * (k - 1) + a;
                        col.w[col.n++] = B[3 * a] * Rd[0] + B[3 * a + 1] * Rd[1] + B[3 * a + 2] * Rd[2];
                    }
                if (q == 3) {   // the phase also maps to its nuisance phase
                    col.row[col.n] = dd.o_ph + (coherent ? k : j * Kt + k);
                    col.w[col.n++] = 1.0;
                }
                gc[q * Kt + k] = col;
            }
            GCol cm;
            cm.n = 1; cm.row[0] = dd.o_a + j * Kt + k; cm.w[0] = 1.0;
            gc[4 * Kt + k] = cm;
        }
        if (tid == 0) { GCol ce; ce.n = 1; ce.row[0] = dd.o_eta; ce.w[0] = 1.0; gc[Lg] = ce; }
        for (int t = tid; t < L * L; t += blockDim.x) Jch[t] = 0.0;
        __syncthreads();
        // J_ch = (2/eta) Re(D^H D) over chunks of elements
        for (int e0 = 0; e0 < Nz; e0 += PCRLB_CH) {
            const int ne = min(PCRLB_CH, Nz - e0);
            for (int t = tid; t < ne * Kt; t += blockDim.x) {
                const int e = t / Kt, k = t - e * Kt;
                const int kk = e0 + e, f = kk / Nm, ym = kk - f * Nm, y = ym / G.Mz, mm = ym - y * G.Mz;
                const double tau = geo[8 * k], th = geo[8 * k + 1], az = geo[8 * k + 2];
                const double sth = sin(th), cth = cos(th), saz = sin(az), caz = cos(az);
                // unit-modulus response and its derivatives (Sec. S-VII-A)
                const double2 a = cisd(-G.f[f] * tau + (G.py[y] * sth * saz + G.pz[mm] * cth) / lam);
                const double dth = 2.0 * M_PI / lam * (G.py[y] * cth * saz - G.pz[mm] * sth);
                const double daz = 2.0 * M_PI / lam * G.py[y] * sth * caz;
                const double dtau = -2.0 * M_PI * G.f[f];
                const double2 r = make_double2(rho[2 * k], rho[2 * k + 1]);
                const double mod = sqrt(r.x * r.x + r.y * r.y);
                const double2 ra = zmul(r, a);
                const double2 ja = make_double2(-ra.y, ra.x);              // j rho a
                double2* row = Dc + (size_t)e * Lg;
                row[k] = make_double2(dth * ja.x, dth * ja.y);            // rho d a / d theta = j dth rho a
                row[Kt + k] = make_double2(daz * ja.x, daz * ja.y);
                row[2 * Kt + k] = make_double2(dtau * ja.x, dtau * ja.y);
                row[3 * Kt + k] = ja;
                const double2 u = mod > 0.0 ? make_double2(r.x / mod, r.y / mod) : make_double2(1.0, 0.0);
                row[4 * Kt + k] = zmul(u, a);                               // e^{j phi} a
            }
            __syncthreads();
            for (int t = tid; t < Lg * Lg; t += blockDim.x) {
                const int u = t / Lg, v = t - u * Lg;
                double acc = 0.0;
                for (int e = 0; e < ne; ++e) {
                    const double2 a = Dc[(size_t)e * Lg + u], b = Dc[(size_t)e * Lg + v];
                    acc += a.x * b.x + a.y * b.y;                           // Re(conj(a) b)
                }
                Jch[u * L + v] += 2.0 / eta * acc;
            }
            __syncthreads();
        }
        if (tid == 0) {
            Jch[Lg * L + Lg] = Nz / (eta * eta);
            // G's nonzeros grouped by global row (counting sort; local index order kept)
            for (int a = 0; a <= dd.dim; ++a) roff[a] = 0;
            for (int u = 0; u < L; ++u)
                for (int i = 0; i < gc[u].n; ++i) ++roff[gc[u].row[i] + 1];
            for (int a = 0; a < dd.dim; ++a) roff[a + 1] += roff[a];
            for (int u = 0; u < L; ++u)
                for (int i = 0; i < gc[u].n; ++i) {
                    const int a = gc[u].row[i];
                    int q = roff[a];
                    while (q < roff[a + 1] && lu[q] >= 0) ++q;   // first free slot of the row
                    lu[q] = u;
                    lw[q] = gc[u].w[i];
                }
        }
        __syncthreads();
        // fim += G J_ch G^T: entry (a, b) = sum over the nonzeros of rows a and b
        for (int t = tid; t < dd.dim * dd.dim; t += blockDim.x) {
            const int a = t / dd.dim, b = t - a * dd.dim;
            double acc = 0.0;
            for (int qa = roff[a]; qa < roff[a + 1]; ++qa)
                for (int qb = roff[b]; qb < roff[b + 1]; ++qb) acc += lw[qa] * Jch[lu[qa] * L + lu[qb]] * lw[qb];
            fim[t] += acc;
        }
        __syncthreads();
        for (int t = tid; t < 7 * L; t += blockDim.x) lu[t] = -1;
    }
}

__global__ void k_pcrlb_mean(int M, int n2, const double* __restrict__ fims, double* __restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n2) return;
    double acc = 0.0;
    for (int m = 0; m < M; ++m) acc += fims[(size_t)m * n2 + t];
    out[t] = acc / M;
}

// in-place inverse of the SPD matrix A (n x n, row-major) by Cholesky, one block; W: n x n scratch
__device__ void spd_inverse(double* A, double* W, int n, int* fail) {
    const int tid = threadIdx.x, nt = blockDim.x;
    // A = L L^T in the lower triangle of W
    for (int t = tid; t < n * n; t += nt) W[t] = A[t];
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (tid == 0) {
            const double d = W[k * n + k];
            if (!(d > 0.0)) *fail = 1;
            W[k * n + k] = d > 0.0 ? sqrt(d) : 1.0;
        }
        __syncthreads();
        const double lkk = W[k * n + k];
        for (int i = k + 1 + tid; i < n; i += nt) W[i * n + k] /= lkk;
        __syncthreads();
        for (int t = tid; t < (n - k - 1) * (n - k - 1); t += nt) {
            const int i = k + 1 + t / (n - k - 1), c = k + 1 + t % (n - k - 1);
            if (c <= i) W[i * n + c] -= W[i * n + k] * W[c * n + k];
        }
        __syncthreads();
    }
    // A^-1 = L^-T L^-1: column c of the inverse solves L y = e_c, L^T x = y (thread per column)
    for (int c = tid; c < n; c += nt) {
        for (int i = 0; i < n; ++i) {   // forward: y stored in A[i * n + c]
            double v = (i == c) ? 1.0 : 0.0;
            for (int q = 0; q < i; ++q) v -= W[i * n + q] * A[q * n + c];
            A[i * n + c] = v / W[i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double v = A[i * n + c];
            for (int q = i + 1; q < n; ++q) v -= W[q * n + i] * A[q * n + c];
            A[i * n + c] = v / W[i * n + i];
        }
    }
    __syncthreads();
}

// J_{n|n} = J_B,n + J_{n|n-1}; P_n = J_{n|n}^-1; J_{n+1|n} = (F P_n F^T + Q)^-1
__global__ void __launch_bounds__(256) k_pcrlb_recursion(int n, int N, int K, const double* __restrict__ F,
                                                         const double* __restrict__ Q, const double* __restrict__ J10,
                                                         const double* __restrict__ Jsnap, double* __restrict__ work,
                                                         double* __restrict__ peb, double* __restrict__ meb, int* fail) {
    const int tid = threadIdx.x, nt = blockDim.x;
    double* Jp = work;                 // J_{n|n-1}
    double* A = work + n * n;          // J_{n|n}, then P_n
    double* W = work + 2 * n * n;      // scratch
    double* T = work + 3 * n * n;      // F P
    for (int t = tid; t < n * n; t += nt) Jp[t] = J10[t];
    __syncthreads();
    for (int s = 0; s < N; ++s) {
        const double* Jb = Jsnap + (size_t)s * n * n;
        for (int t = tid; t < n * n; t += nt) A[t] = Jb[t] + Jp[t];
        __syncthreads();
        spd_inverse(A, W, n, fail);   // A = P_n
        if (tid == 0) {
            peb[s] = sqrt(A[0] + A[n + 1] + A[2 * n + 2]);
            for (int k = 0; k < K; ++k) {
                const int o = 6 + 3 * k;
                meb[(size_t)s * K + k] = sqrt(A[o * n + o] + A[(o + 1) * n + o + 1] + A[(o + 2) * n + o + 2]);
            }
        }
        // Jp = (F P F^T + Q)^-1
        for (int t = tid; t < n * n; t += nt) {
            const int i = t / n, c = t - i * n;
            double v = 0.0;
            for (int q = 0; q < n; ++q) v += F[i * n + q] * A[q * n + c];
            T[t] = v;
        }
        __syncthreads();
        for (int t = tid; t < n * n; t += nt) {
            const int i = t / n, c = t - i * n;
            double v = Q[t];
            for (int q = 0; q < n; ++q) v += T[i * n + q] * F[c * n + q];
            Jp[t] = v;
        }
        __syncthreads();
        spd_inverse(Jp, W, n, fail);
    }
}

size_t pcrlb_fim_smem(int K, int J, bool coherent) {
    const PcrlbDims dd(K, J, coherent);
    const size_t Lg = 5 * (size_t)dd.Kt, L = dd.L;
    return PCRLB_CH * Lg * sizeof(double2) + L * L * sizeof(double) + L * sizeof(GCol) + 8 * dd.Kt * sizeof(double) +
           7 * L * sizeof(double) + 7 * L * sizeof(int) + (dd.dim + 1) * sizeof(int);
}

}  // namespace bp

using namespace bp;

namespace {
struct DevBufs {
    std::vector<void*> p;
    ~DevBufs() { for (void* q : p) cudaFree(q); }
    template <typename T> T* get(size_t n) {
        void* q = nullptr;
        if (cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) return nullptr;
        p.push_back(q);
        return static_cast<T*>(q);
    }
};
}  // namespace

extern "C" {

bp_status bp_pcrlb_fim(const bp_geometry* geom, int K, int coherent, int M, const double* x, const double* sfv,
                       const double* rho, double eta, double* fim, void* cuda_stream) {
    if (validate_geom(geom) != BP_OK || K < 0 || K > PCRLB_KMAX || M < 1 || !x || !rho || !fim || (K > 0 && !sfv) ||
        !(eta > 0.0))
        return BP_ERR_INVALID_ARG;
    DevGeom G;
    fill_geom(G, geom);
    const PcrlbDims dd(K, G.J, coherent != 0);
    const size_t n2 = (size_t)dd.dim * dd.dim;
    const size_t smem = pcrlb_fim_smem(K, G.J, coherent != 0);
    if (smem > (size_t)smem_optin()) return BP_ERR_CAPACITY;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    DevBufs b;
    double* dx = b.get<double>((size_t)M * 6);
    double* ds = b.get<double>((size_t)M * K * 3);
    double* dr = b.get<double>((size_t)M * G.J * (K + 1) * 2);
    double* dfims = b.get<double>((size_t)M * n2);
    double* dout = b.get<double>(n2);
    if (!dx || !ds || !dr || !dfims || !dout) return BP_ERR_CUDA;
    bool ok = cudaMemcpyAsync(dx, x, (size_t)M * 6 * sizeof(double), cudaMemcpyHostToDevice, st) == cudaSuccess &&
              (K == 0 || cudaMemcpyAsync(ds, sfv, (size_t)M * K * 3 * sizeof(double), cudaMemcpyHostToDevice, st) == cudaSuccess) &&
              cudaMemcpyAsync(dr, rho, (size_t)M * G.J * (K + 1) * 2 * sizeof(double), cudaMemcpyHostToDevice, st) == cudaSuccess;
    if (!ok) return BP_ERR_CUDA;
    smem_allow_max((const void*)k_pcrlb_fim);
    k_pcrlb_fim<<<M, 256, smem, st>>>(G, K, coherent != 0, dx, ds, dr, eta, dfims);
    k_pcrlb_mean<<<(unsigned)((n2 + 255) / 256), 256, 0, st>>>(M, (int)n2, dfims, dout);
    if (cudaMemcpyAsync(fim, dout, n2 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return BP_ERR_CUDA;
    return BP_OK;
}

bp_status bp_pcrlb_recursion(int dim, int N, int K, const double* F, const double* Q, const double* J10,
                             const double* Jsnap, double* peb, double* meb, void* cuda_stream) {
    if (dim < 6 + 3 * K || N < 1 || K < 0 || !F || !Q || !J10 || !Jsnap || !peb || (K > 0 && !meb) || dim > 4096)
        return BP_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const size_t n2 = (size_t)dim * dim;
    DevBufs b;
    double* dF = b.get<double>(n2);
    double* dQ = b.get<double>(n2);
    double* dJ10 = b.get<double>(n2);
    double* dJs = b.get<double>((size_t)N * n2);
    double* dw = b.get<double>(4 * n2);
    double* dpeb = b.get<double>(N);
    double* dmeb = b.get<double>((size_t)N * std::max(K, 1));
    int* dfail = b.get<int>(1);
    if (!dF || !dQ || !dJ10 || !dJs || !dw || !dpeb || !dmeb || !dfail) return BP_ERR_CUDA;
    bool ok = cudaMemcpyAsync(dF, F, n2 * 8, cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(dQ, Q, n2 * 8, cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(dJ10, J10, n2 * 8, cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(dJs, Jsnap, (size_t)N * n2 * 8, cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemsetAsync(dfail, 0, sizeof(int), st) == cudaSuccess;
    if (!ok) return BP_ERR_CUDA;
    k_pcrlb_recursion<<<1, 256, 0, st>>>(dim, N, K, dF, dQ, dJ10, dJs, dw, dpeb, dmeb, dfail);
    int fail = 0;
    ok = cudaMemcpyAsync(peb, dpeb, (size_t)N * 8, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
         (K == 0 || cudaMemcpyAsync(meb, dmeb, (size_t)N * K * 8, cudaMemcpyDeviceToHost, st) == cudaSuccess) &&
         cudaMemcpyAsync(&fail, dfail, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
         cudaStreamSynchronize(st) == cudaSuccess && cudaGetLastError() == cudaSuccess;
    if (!ok) return BP_ERR_CUDA;
    return fail ? BP_ERR_NUMERIC : BP_OK;
}

}  // extern "C"
