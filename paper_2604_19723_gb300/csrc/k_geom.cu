// Per-(particle, feature, PA) geometry of the current prediction, once per step:
// virtual anchor and Householder mirror (eq. posPA-SB, house), local vector
// r' = R^T H (p - p_va) (eq. rangep), its length and direction, in float-float
// arithmetic on the FP32 pipe (about 44 significant bits; the particle positions are
// FP32, the PA positions and rotations FP32 pairs).  The likelihood and table kernels
// rebuild the steering vectors from these records in FP32 (factors_from_geo), so they
// carry no such work.
#include "bp_internal.cuh"
#include "bp_kernels.cuh"

namespace bp {

__device__ inline ff ffx(float a) { return ff{a, 0.f}; }
__device__ inline ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }
__device__ inline ff ff_twice(ff x) { return ff{2.0f * x.hi, 2.0f * x.lo}; }   // exact
__device__ inline ff ff_mulf(ff x, float b) {                                    // x b
    const float p = __fmul_rn(x.hi, b);
    const float e = fmaf(x.lo, b, fmaf(x.hi, b, -p));
    ff r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
}
__device__ inline ff ff_sqrt(ff x) {   // one correction of the FP32 root: s + (x - s^2) / (2 s)
    const float s = sqrtf(x.hi);
    const ff r = ff_sub(x, ff_prod(s, s));
    ff out;
    fast_two_sum(s, __fdiv_rn(r.hi, 2.0f * s), out.hi, out.lo);
    return out;
}

__global__ void k_geom(DevGeom G, DevParams Pm, DevState D, int S) {
    const int P = Pm.P, J = G.J;
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)S * J * P) return;
    const int p = (int)(idx % P);
    const int sj = (int)(idx / P);
    const int s = sj / J, j = sj - s * J;
    const float* x = D.x[D.cur];
    const float* ph = D.phi[D.cur] + (size_t)s * 6 * P;
    const float px = x[p], py = x[P + p], pz = x[2 * P + p];
    const ff ax{G.pa_h[j][0], G.pa_l[j][0]}, ay{G.pa_h[j][1], G.pa_l[j][1]}, az{G.pa_h[j][2], G.pa_l[j][2]};
    ff rx, ry, rz;
    if (s == 0) {   // LoS: r = p - p_pa
        rx = ff_sub(ffx(px), ax); ry = ff_sub(ffx(py), ay); rz = ff_sub(ffx(pz), az);
    } else {        // PF s: mirror the PA through the plane at p_sfv with normal p_sfv
        const float sx = ph[p], sy = ph[P + p], sz = ph[2 * P + p];
        const ff nn = ff_add(ff_add(ff_prod(sx, sx), ff_prod(sy, sy)), ff_prod(sz, sz));
        const ff as = ff_add(ff_add(ff_mulf(ax, sx), ff_mulf(ay, sy)), ff_mulf(az, sz));
        const ff coef = ff_sub(ff_div(ff_twice(as), nn), ffx(1.0f));             // 2 a.s / |s|^2 - 1
        const ff vx = ff_sub(ax, ff_mulf(coef, sx)), vy = ff_sub(ay, ff_mulf(coef, sy)),
                 vz = ff_sub(az, ff_mulf(coef, sz));                                // virtual anchor
        const ff qx = ff_sub(ffx(px), vx), qy = ff_sub(ffx(py), vy), qz = ff_sub(ffx(pz), vz);
        const ff sq = ff_add(ff_add(ff_mulf(qx, sx), ff_mulf(qy, sy)), ff_mulf(qz, sz));
        const ff t = ff_div(ff_twice(sq), nn);                                      // Householder H q
        rx = ff_sub(qx, ff_mulf(t, sx)); ry = ff_sub(qy, ff_mulf(t, sy)); rz = ff_sub(qz, ff_mulf(t, sz));
    }
    auto Rk = [&](int k) { return ff{G.R_h[j][k], G.R_l[j][k]}; };
    const ff lx = ff_add(ff_add(ff_mul(Rk(0), rx), ff_mul(Rk(3), ry)), ff_mul(Rk(6), rz));
    const ff ly = ff_add(ff_add(ff_mul(Rk(1), rx), ff_mul(Rk(4), ry)), ff_mul(Rk(7), rz));
    const ff lz = ff_add(ff_add(ff_mul(Rk(2), rx), ff_mul(Rk(5), ry)), ff_mul(Rk(8), rz));
    const ff d = ff_sqrt(ff_add(ff_add(ff_mul(lx, lx), ff_mul(ly, ly)), ff_mul(lz, lz)));
    const ff uy = ff_div(ly, d), uz = ff_div(lz, d);
    D.geo[idx] = make_float4(d.hi, d.lo, uy.hi, uz.hi);
    D.geo_lo[idx] = make_float2(uy.lo, uz.lo);
}

void launch_geom(const DevGeom& G, const DevParams& Pm, const DevState& D, int S, cudaStream_t st) {
    const long n = (long)S * G.J * Pm.P;
    k_geom<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(G, Pm, D, S);
}

}  // namespace bp
