// Per-(particle, feature, PA) geometry of the current prediction, once per step.
// FP64: virtual anchor and Householder mirror (eq. posPA-SB, house), local
// vector r' = R^T H (p - p_va) (eq. rangep), its length and direction.  The
// likelihood and table kernels rebuild the steering vectors from these
// records in FP32 (factors_from_geo), so they carry no FP64 work.
#include "bp_internal.cuh"
#include "bp_kernels.cuh"

namespace bp {

__global__ void k_geom(DevGeom G, DevParams Pm, DevState D, int S) {
    const int P = Pm.P, J = G.J;
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)S * J * P) return;
    const int p = (int)(idx % P);
    const int sj = (int)(idx / P);
    const int s = sj / J, j = sj - s * J;
    const float* x = D.x[D.cur];
    const float* ph = D.phi[D.cur] + (size_t)s * 6 * P;
    const PathGeo pg = path_geo(G, j, x[p], x[P + p], x[2 * P + p], ph[p], ph[P + p], ph[2 * P + p], s == 0);
    const float dh = (float)pg.d;
    const float dl = (float)(pg.d - (double)dh);
    const float uyh = (float)pg.uy, uzh = (float)pg.uz;
    D.geo[idx] = make_float4(dh, dl, uyh, uzh);
    D.geo_lo[idx] = make_float2((float)(pg.uy - (double)uyh), (float)(pg.uz - (double)uzh));
}

void launch_geom(const DevGeom& G, const DevParams& Pm, const DevState& D, int S, cudaStream_t st) {
    const long n = (long)S * G.J * Pm.P;
    k_geom<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(G, Pm, D, S);
}

}  // namespace bp
