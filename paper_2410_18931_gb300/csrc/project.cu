// Per-Gaussian projection (forward) and its gradient chain (backward).
//
// Forward, one thread per Gaussian, looping over the views so the parameters
// are read from HBM once per call:
//   Sec. 3 Eq. 3   Sigma_3D = R S S^t R^t          (R from the normalised quaternion)
//   Sec. 3 Eq. 5   Sigma_2D = J W Sigma_3D W^t J^t  (+ 0.3 I, J clamped at 1.3 tan(fov))
//   Sec. 3 Eq. 4   c = max(0, Y(dir) . H + 0.5)
//   Eq. 11 / Eq. 3 u = Y(dir) . H^alpha (unclamped) or sigmoid(o)
//   Eqs. 8-10      w(d) with d = camera z
// and writes the 48-byte render record {mu, qs, qw, qd, u w, c u w, extents}
// with the footprint's quadratic form, prescaled by log2(e)/2, as the sum of
// squares q' = (qs dy + qw dx)^2 + qd dx^2.
//
// Backward, one thread per Gaussian: the render backward's record of each
// (view, Gaussian) holds moments of dL/dq' in that sum-of-squares frame plus
// d/d(u w) and d/d(c u w); they are chained to the mean, the 2D covariance
// (in factored form), the colour and opacity SH, the depth weight and the
// stored parameters, summed over views.
//
// The 2D covariance is formed as T T^t with T = J W R S (2x3), so its
// determinant is the squared norm of the cross product of T's rows (plus the
// dilation terms): a sum of squares with no cancellation.  For strongly
// anisotropic footprints (det < 1e-3 a c) the conic is recomputed in FP64
// from the same rows.
#include "wsr_launch.h"

namespace wsr {
namespace {

struct Geom {
    float tx, ty, tz;
    float M[9];            // W R diag(s), row-major
    float J00, J02, J11, J12;
    float rxc, ryc;        // clamped x/z and y/z
    bool freex, freey;     // not clamped
    float r0[3], r1[3];    // rows of T = J W R S
    float a, b, c;         // Sigma_2D with dilation
    float A, B, C;         // conic
    // the same quadratic form as a sum of squares, prescaled by log2(e)/2:
    // q' = (qs dy + qw dx)^2 + qd dx^2, i.e. q = (a/det)(dy - (b/a) dx)^2 + dx^2 / a
    float qs, qw, qd;
};

__device__ __forceinline__ void geometry(const View& V, const float* Rg, const float* s, float px,
                                         float py, float pz, Geom& G) {
    G.tx = V.R[0] * px + V.R[1] * py + V.R[2] * pz + V.T[0];
    G.ty = V.R[3] * px + V.R[4] * py + V.R[5] * pz + V.T[1];
    G.tz = V.R[6] * px + V.R[7] * py + V.R[8] * pz + V.T[2];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            G.M[3 * r + c] =
                (V.R[3 * r] * Rg[c] + V.R[3 * r + 1] * Rg[3 + c] + V.R[3 * r + 2] * Rg[6 + c]) * s[c];
    const float iz = 1.0f / G.tz;
    const float ux = G.tx * iz, uy = G.ty * iz;
    G.rxc = fminf(fmaxf(ux, -V.limx), V.limx);
    G.ryc = fminf(fmaxf(uy, -V.limy), V.limy);
    G.freex = (ux >= -V.limx) && (ux <= V.limx);
    G.freey = (uy >= -V.limy) && (uy <= V.limy);
    G.J00 = V.fx * iz;
    G.J02 = -V.fx * G.rxc * iz;
    G.J11 = V.fy * iz;
    G.J12 = -V.fy * G.ryc * iz;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        G.r0[k] = G.J00 * G.M[k] + G.J02 * G.M[6 + k];
        G.r1[k] = G.J11 * G.M[3 + k] + G.J12 * G.M[6 + k];
    }
    const float a0 = G.r0[0] * G.r0[0] + G.r0[1] * G.r0[1] + G.r0[2] * G.r0[2];
    const float c0 = G.r1[0] * G.r1[0] + G.r1[1] * G.r1[1] + G.r1[2] * G.r1[2];
    const float b0 = G.r0[0] * G.r1[0] + G.r0[1] * G.r1[1] + G.r0[2] * G.r1[2];
    const float x0 = G.r0[1] * G.r1[2] - G.r0[2] * G.r1[1];
    const float x1 = G.r0[2] * G.r1[0] - G.r0[0] * G.r1[2];
    const float x2 = G.r0[0] * G.r1[1] - G.r0[1] * G.r1[0];
    G.a = a0 + kDilation;
    G.c = c0 + kDilation;
    G.b = b0;
    const float det = (x0 * x0 + x1 * x1 + x2 * x2) + kDilation * (a0 + c0) + kDilation * kDilation;
    if (det < 1e-3f * G.a * G.c) {
        // strongly anisotropic footprint: conic in FP64 from the same rows
        const double p0 = G.r0[0], p1 = G.r0[1], p2 = G.r0[2];
        const double q0 = G.r1[0], q1 = G.r1[1], q2 = G.r1[2];
        const double ad = p0 * p0 + p1 * p1 + p2 * p2, cd = q0 * q0 + q1 * q1 + q2 * q2;
        const double bd = p0 * q0 + p1 * q1 + p2 * q2;
        const double y0 = p1 * q2 - p2 * q1, y1 = p2 * q0 - p0 * q2, y2 = p0 * q1 - p1 * q0;
        const double dd = (y0 * y0 + y1 * y1 + y2 * y2) + 0.3 * (ad + cd) + 0.09;
        G.A = (float)((cd + 0.3) / dd);
        G.B = (float)(-bd / dd);
        G.C = (float)((ad + 0.3) / dd);
        const double k = (double)kHalfLog2e, a_ = ad + 0.3;
        const double qs = sqrt(k * a_ / dd);
        G.qs = (float)qs;
        G.qw = (float)(-(bd / a_) * qs);
        G.qd = (float)(k / a_);
    } else {
        const float id = 1.0f / det;
        G.A = G.c * id;
        G.B = -G.b * id;
        G.C = G.a * id;
        G.qs = sqrtf(kHalfLog2e * G.a * id);
        G.qw = -(G.b / G.a) * G.qs;
        G.qd = kHalfLog2e / G.a;
    }
}

template <int DEG, bool VD, bool RED>
struct Params {
    static constexpr int K = (DEG + 1) * (DEG + 1);
    float p[3], ls[3], q[4];
    float H[K * 3];
    float Ha[VD ? K : 1];
    float lcv;
};

template <int DEG, bool VD, bool RED>
__device__ __forceinline__ void load_params(const GaussPtrs& g, long long i, int wkind,
                                            Params<DEG, VD, RED>& P) {
    using sq_t = typename Store<RED>::sq_t;
    using sh_t = typename Store<RED>::sh_t;
    constexpr int K = Params<DEG, VD, RED>::K;
    P.p[0] = __ldg(g.means + 3 * i);
    P.p[1] = __ldg(g.means + 3 * i + 1);
    P.p[2] = __ldg(g.means + 3 * i + 2);
    load_n<sq_t, 3>(reinterpret_cast<const sq_t*>(g.log_scales) + 3 * i, P.ls);
    load_n<sq_t, 4>(reinterpret_cast<const sq_t*>(g.quats) + 4 * i, P.q);
    load_n<sh_t, K * 3>(reinterpret_cast<const sh_t*>(g.sh) + (long long)K * 3 * i, P.H);
    if constexpr (VD) {
        load_n<sh_t, K>(reinterpret_cast<const sh_t*>(g.opacity) + (long long)K * i, P.Ha);
    } else {
        load_n<sh_t, 1>(reinterpret_cast<const sh_t*>(g.opacity) + i, P.Ha);
    }
    P.lcv = (wkind == WSR_WEIGHT_LC) ? __ldg(g.lc_v + i) : 0.0f;
}

// Normalised quaternion, rotation and scales.
__device__ __forceinline__ void rot_scale(const float* qr, const float* ls, float* qn, float& qlen,
                                          float* Rg, float* s) {
    const float n2 = qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3];
    qlen = sqrtf(n2);
    const float inv = 1.0f / qlen;
#pragma unroll
    for (int k = 0; k < 4; ++k) qn[k] = qr[k] * inv;
    quat_rot(qn[0], qn[1], qn[2], qn[3], Rg);
#pragma unroll
    for (int k = 0; k < 3; ++k) s[k] = expf(ls[k]);
}

// The depth factor of the weight (Eqs. 8-10): w = factor for DIR and EXP, w = factor * v_i for LC.
// A Gaussian is culled only where the factor is 0 (LC beyond sigma, EXP underflow): there neither
// Eq. 7 nor its gradient depends on it.  Where only v_i is 0, w = 0 but dw/dv_i is not, so it stays.
__device__ __forceinline__ float depth_factor(int kind, float d, float sigma, float beta) {
    if (kind == WSR_WEIGHT_EXP) return expf(-sigma * powf(d, beta));
    if (kind == WSR_WEIGHT_LC) return fmaxf(0.0f, 1.0f - d / sigma);
    return 1.0f;
}

template <int DEG, bool VD, bool RED>
__global__ void __launch_bounds__(256) k_project(const GaussPtrs g, const Views vs, const WeightDev wd,
                                                 float4* __restrict__ rec) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    Params<DEG, VD, RED> P;
    load_params<DEG, VD, RED>(g, i, wd.kind, P);
    const float sigma = __ldg(wd.params + 0), beta = __ldg(wd.params + 1);
    float qn[4], qlen, Rg[9], s[3];
    rot_scale(P.q, P.ls, qn, qlen, Rg, s);

    for (int v = 0; v < vs.n; ++v) {
        const View& V = vs.v[v];
        float4* o = rec + 3 * ((long long)v * g.n + i);
        const float tz = V.R[6] * P.p[0] + V.R[7] * P.p[1] + V.R[8] * P.p[2] + V.T[2];
        float wf = 0.0f;
        if (tz > V.znear) wf = depth_factor(wd.kind, tz, sigma, beta);
        if (!(tz > V.znear) || wf == 0.0f) {
            // culled: behind the near plane (App. C), or a zero depth factor
            // (LC beyond sigma), which contributes nothing to Eq. 7 or its gradient
            o[0] = make_float4(0.f, 0.f, 0.f, 0.f);
            o[1] = make_float4(0.f, 0.f, 0.f, 0.f);
            o[2] = make_float4(0.f, -1.f, -1.f, tz);
            continue;
        }
        const float w = (wd.kind == WSR_WEIGHT_LC) ? wf * P.lcv : wf;
        Geom G;
        geometry(V, Rg, s, P.p[0], P.p[1], P.p[2], G);
        const float mx = V.fx * G.tx / G.tz + V.cx;
        const float my = V.fy * G.ty / G.tz + V.cy;
        // 3-sigma half extents, slightly widened so that binning stays
        // conservative with respect to the FP32 cutoff test of the renderer
        const float rx = 3.0f * sqrtf(G.a) * 1.0001f + 0.01f;
        const float ry = 3.0f * sqrtf(G.c) * 1.0001f + 0.01f;

        float dx = P.p[0] - V.campos[0], dy = P.p[1] - V.campos[1], dz = P.p[2] - V.campos[2];
        const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
        dx *= il; dy *= il; dz *= il;
        float Y[K];
        sh_basis<DEG>(dx, dy, dz, Y);
        float col[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float r = 0.0f;
#pragma unroll
            for (int k = 0; k < K; ++k) r += Y[k] * P.H[3 * k + ch];
            col[ch] = fmaxf(r + 0.5f, 0.0f);
        }
        float u;
        if constexpr (VD) {
            u = 0.0f;
#pragma unroll
            for (int k = 0; k < K; ++k) u += Y[k] * P.Ha[k];
        } else {
            u = 1.0f / (1.0f + expf(-P.Ha[0]));
        }
        const float uw = u * w;
        o[0] = make_float4(mx, my, G.qs, G.qw);
        o[1] = make_float4(G.qd, uw, col[0] * uw, col[1] * uw);
        o[2] = make_float4(col[2] * uw, rx, ry, G.tz);
    }
}

// ---------------------------------------------------------------------------
// Backward chain: grad record {dmu, dA, dB, dC, d(uw), d(c uw)} per view ->
// parameters.  Recomputes every forward intermediate from the parameters.
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ void store_n(float* __restrict__ p, const float* v) {
    if constexpr ((N * 4) % 16 == 0) {
        float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
        for (int k = 0; k < N / 4; ++k) q[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < N; ++k) p[k] = v[k];
    }
}

// ONE: a single view.  Its SH and opacity-SH gradients are final as soon as
// they are formed, so they are stored there and neither they nor the SH
// coefficients stay live through the geometry chain (about 60 registers
// fewer: three blocks of 128 per SM instead of two).
template <int DEG, bool VD, bool RED, bool ONE>
__global__ void __launch_bounds__(128, ONE ? 3 : 1) k_project_bwd(const GaussPtrs g, const Views vs, const WeightDev wd,
                                                     const float* __restrict__ grec, const wsr_grads out,
                                                     float* __restrict__ det_sb) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    float gsig = 0.0f, gbeta = 0.0f;
    // det_sb != nullptr: deterministic mode (fixed-point records, a bounded grid striding over the
    // Gaussians, sigma/beta summed per block in a fixed order into det_sb)
    auto body = [&](const long long i) {
        Params<DEG, VD, RED> P;
        load_params<DEG, VD, RED>(g, i, wd.kind, P);
        const float sigma = __ldg(wd.params + 0), beta = __ldg(wd.params + 1);
        float qn[4], qlen, Rg[9], s[3];
        rot_scale(P.q, P.ls, qn, qlen, Rg, s);

        float gp[3] = {0.f, 0.f, 0.f}, gs[3] = {0.f, 0.f, 0.f}, gR[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) gR[e] = 0.f;
        float gH[K * 3];
#pragma unroll
        for (int e = 0; e < K * 3; ++e) gH[e] = 0.f;
        float gHa[VD ? K : 1];
#pragma unroll
        for (int e = 0; e < (VD ? K : 1); ++e) gHa[e] = 0.f;
        float glcv = 0.f;
        bool sh_stored = false;

        const int nv = ONE ? 1 : vs.n;
        for (int v = 0; v < nv; ++v) {
            const View& V = vs.v[v];
            float g9[9];
            bool any = false;
            if (det_sb == nullptr) {
                const float* gr = grec + WSR_GRAD_RECORD_FLOATS * ((long long)v * g.n + i);
#pragma unroll
                for (int e = 0; e < 9; ++e) {
                    g9[e] = __ldg(gr + e);
                    any |= (g9[e] != 0.0f);
                }
            } else {
                // 9 int64 sums in units of 2^(e - kDetBits), 2^e above the term's bound (stored beside them)
                const float* gr = grec + kDetRecordFloats * ((long long)v * g.n + i);
                const long long* sums = reinterpret_cast<const long long*>(gr);
                const int* mag = reinterpret_cast<const int*>(gr + 18);
#pragma unroll
                for (int c = 0; c < 9; ++c) {
                    const float m = __int_as_float(__ldg(mag + c));
                    float val = 0.0f;
                    if (m > 0.0f) {
                        int e;
                        frexpf(m, &e);
                        val = (float)ldexp((double)__ldg(sums + c), e - kDetBits);
                    }
                    g9[c] = val;
                    any |= (val != 0.0f);
                }
            }
            if (!any) continue;
            const float tz0 = V.R[6] * P.p[0] + V.R[7] * P.p[1] + V.R[8] * P.p[2] + V.T[2];
            if (!(tz0 > V.znear)) continue;
            const float wf = depth_factor(wd.kind, tz0, sigma, beta);
            if (wf == 0.0f) continue;
            const float w = (wd.kind == WSR_WEIGHT_LC) ? wf * P.lcv : wf;
            Geom G;
            geometry(V, Rg, s, P.p[0], P.p[1], P.p[2], G);
            const float tx = G.tx, ty = G.ty, tz = G.tz;

            float vx = P.p[0] - V.campos[0], vy = P.p[1] - V.campos[1], vz = P.p[2] - V.campos[2];
            const float il = rsqrtf(vx * vx + vy * vy + vz * vz);
            const float dx = vx * il, dy = vy * il, dz = vz * il;
            float Y[K];
            sh_basis<DEG>(dx, dy, dz, Y);
            float raw[3], col[3];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                float r = 0.0f;
#pragma unroll
                for (int k = 0; k < K; ++k) r += Y[k] * P.H[3 * k + ch];
                raw[ch] = r;
                col[ch] = fmaxf(r + 0.5f, 0.0f);
            }
            float u;
            if constexpr (VD) {
                u = 0.0f;
#pragma unroll
                for (int k = 0; k < K; ++k) u += Y[k] * P.Ha[k];
            } else {
                u = 1.0f / (1.0f + expf(-P.Ha[0]));
            }
            const float uw = u * w;

            // Eq. 7 record terms -> colour, opacity, weight
            const float gcuw[3] = {g9[6], g9[7], g9[8]};
            const float guw = g9[5] + gcuw[0] * col[0] + gcuw[1] * col[1] + gcuw[2] * col[2];
            const float gu = guw * w, gw = guw * u;
            float graw[3];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) graw[ch] = (raw[ch] + 0.5f > 0.0f) ? gcuw[ch] * uw : 0.0f;
            float wk[K];
            if constexpr (ONE) {
                float gHv[K * 3];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    gHv[3 * k + 0] = graw[0] * Y[k];
                    gHv[3 * k + 1] = graw[1] * Y[k];
                    gHv[3 * k + 2] = graw[2] * Y[k];
                    wk[k] = graw[0] * P.H[3 * k] + graw[1] * P.H[3 * k + 1] + graw[2] * P.H[3 * k + 2];
                }
                if (out.sh) store_n<K * 3>(out.sh + (long long)K * 3 * i, gHv);
                if constexpr (VD) {
                    float gHav[K];
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        gHav[k] = gu * Y[k];
                        wk[k] += gu * P.Ha[k];
                    }
                    if (out.opacity) store_n<K>(out.opacity + (long long)K * i, gHav);
                } else {
                    if (out.opacity) out.opacity[i] = gu * u * (1.0f - u);
                }
                sh_stored = true;
            } else {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    gH[3 * k + 0] += graw[0] * Y[k];
                    gH[3 * k + 1] += graw[1] * Y[k];
                    gH[3 * k + 2] += graw[2] * Y[k];
                    wk[k] = graw[0] * P.H[3 * k] + graw[1] * P.H[3 * k + 1] + graw[2] * P.H[3 * k + 2];
                }
                if constexpr (VD) {
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        gHa[k] += gu * Y[k];
                        wk[k] += gu * P.Ha[k];
                    }
                } else {
                    gHa[0] += gu * u * (1.0f - u);
                }
            }
            // direction dir = (p - f)/|p - f|: tangential part of the SH gradient
            float gdx = 0.f, gdy = 0.f, gdz = 0.f;
            sh_grad_dot<DEG>(dx, dy, dz, wk, gdx, gdy, gdz);
            const float dd = dx * gdx + dy * gdy + dz * gdz;
            gp[0] += (gdx - dx * dd) * il;
            gp[1] += (gdy - dy * dd) * il;
            gp[2] += (gdz - dz * dd) * il;

            // depth weight, d = t_z
            float gt[3] = {0.f, 0.f, 0.f};
            if (wd.kind == WSR_WEIGHT_EXP) {
                const float db = powf(tz, beta);
                gsig += gw * (-db) * w;
                gbeta += gw * (-sigma * db * logf(tz)) * w;
                gt[2] += gw * (-sigma * beta * db / tz) * w;
            } else if (wd.kind == WSR_WEIGHT_LC) {
                const float lin = 1.0f - tz / sigma;
                glcv += gw * lin;
                gsig += gw * P.lcv * tz / (sigma * sigma);
                gt[2] += gw * (-P.lcv / sigma);
            }
            // The record holds moments of gq = dL/dq' over the Gaussian's pixels in the sum-of-squares
            // frame of q' = r^2 + qd dx^2, r = qs dy + qw dx (qs, qw, qd exactly as rendered):
            // Sr = sum gq r, Sx = sum gq dx, Srr = sum gq r^2, Srx = sum gq r dx, Sxx = sum gq dx^2.
            const float Sr = g9[0], Sx = g9[1], Srr = g9[2], Srx = g9[3], Sxx = g9[4];
            const float qs = G.qs, qw = G.qw, qd = G.qd;
            // projected mean: dq'/dmu_x = -2 (r qw + qd dx), dq'/dmu_y = -2 r qs
            const float gmx = -2.0f * fmaf(qw, Sr, qd * Sx), gmy = -2.0f * qs * Sr;
            const float iz = 1.0f / tz, iz2 = iz * iz;
            gt[0] += gmx * V.fx * iz;
            gt[1] += gmy * V.fy * iz;
            gt[2] += -(gmx * V.fx * tx + gmy * V.fy * ty) * iz2;

            // Sigma_2D = T T^t + 0.3 I with rows r0, r1 of T = J W R S.  With v = k Sigma_2D^{-1} d =
            // r w + qd dx e1 (w = (qw, qs), e1 = (1, 0), k = log2(e)/2), dq'/dSigma_2D = -v v^t / k, so
            //   dL/dSigma_2D = -(Srr w w^t + qd Srx (w e1^t + e1 w^t) + qd^2 Sxx e1 e1^t) / k
            // and dL/dT = 2 dL/dSigma_2D T is taken in that factored form: with z = w^t T = qw r0 + qs r1,
            //   dL/dr0 = -2/k (qw P1 + P2),  dL/dr1 = -2/k qs P1,
            //   P1 = Srr z + qd Srx r0,  P2 = qd Srx z + qd^2 Sxx r0.
            // For a thin footprint z is nearly orthogonal to the long axis, so the large Srr terms
            // stay off that axis instead of cancelling there in FP32.
            const float c2 = -2.0f / kHalfLog2e, qsx = qd * Srx, qxx = qd * qd * Sxx;
            float gr0[3], gr1[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float z = fmaf(qw, G.r0[k], qs * G.r1[k]);
                const float P1 = fmaf(Srr, z, qsx * G.r0[k]);
                const float P2 = fmaf(qsx, z, qxx * G.r0[k]);
                gr0[k] = c2 * fmaf(qw, P1, P2);
                gr1[k] = c2 * qs * P1;
            }
            // r0 = J00 m0 + J02 m2,  r1 = J11 m1 + J12 m2  (m_k: rows of M = W R S)
            float gJ00 = 0.f, gJ02 = 0.f, gJ11 = 0.f, gJ12 = 0.f, gM[9];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                gJ00 += gr0[k] * G.M[k];
                gJ02 += gr0[k] * G.M[6 + k];
                gJ11 += gr1[k] * G.M[3 + k];
                gJ12 += gr1[k] * G.M[6 + k];
                gM[k] = G.J00 * gr0[k];
                gM[3 + k] = G.J11 * gr1[k];
                gM[6 + k] = G.J02 * gr0[k] + G.J12 * gr1[k];
            }
            // J(t): J00 = fx/tz, J02 = -fx rx/tz, J11 = fy/tz, J12 = -fy ry/tz
            gt[2] += -(gJ00 * V.fx + gJ11 * V.fy) * iz2 + (gJ02 * V.fx * G.rxc + gJ12 * V.fy * G.ryc) * iz2;
            if (G.freex) {
                gt[0] += -gJ02 * V.fx * iz2;
                gt[2] += gJ02 * V.fx * tx * iz2 * iz;
            }
            if (G.freey) {
                gt[1] += -gJ12 * V.fy * iz2;
                gt[2] += gJ12 * V.fy * ty * iz2 * iz;
            }
            // t = W p + T
#pragma unroll
            for (int k = 0; k < 3; ++k) gp[k] += V.R[k] * gt[0] + V.R[3 + k] * gt[1] + V.R[6 + k] * gt[2];
            // M = W N, N = R diag(s):  gN = W^t gM
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float gN = V.R[r] * gM[c] + V.R[3 + r] * gM[3 + c] + V.R[6 + r] * gM[6 + c];
                    gR[3 * r + c] += gN * s[c];
                    gs[c] += gN * Rg[3 * r + c];
                }
        }

        // rotation <- normalised quaternion <- raw quaternion
        const float w_ = qn[0], x_ = qn[1], y_ = qn[2], z_ = qn[3];
        float gqn[4];
        gqn[0] = -2.f * z_ * gR[1] + 2.f * y_ * gR[2] + 2.f * z_ * gR[3] - 2.f * x_ * gR[5] - 2.f * y_ * gR[6] +
                 2.f * x_ * gR[7];
        gqn[1] = 2.f * y_ * gR[1] + 2.f * z_ * gR[2] + 2.f * y_ * gR[3] - 4.f * x_ * gR[4] - 2.f * w_ * gR[5] +
                 2.f * z_ * gR[6] + 2.f * w_ * gR[7] - 4.f * x_ * gR[8];
        gqn[2] = -4.f * y_ * gR[0] + 2.f * x_ * gR[1] + 2.f * w_ * gR[2] + 2.f * x_ * gR[3] + 2.f * z_ * gR[5] -
                 2.f * w_ * gR[6] + 2.f * z_ * gR[7] - 4.f * y_ * gR[8];
        gqn[3] = -4.f * z_ * gR[0] - 2.f * w_ * gR[1] + 2.f * x_ * gR[2] + 2.f * w_ * gR[3] - 4.f * z_ * gR[4] +
                 2.f * y_ * gR[5] + 2.f * x_ * gR[6] + 2.f * y_ * gR[7];
        const float qd = gqn[0] * qn[0] + gqn[1] * qn[1] + gqn[2] * qn[2] + gqn[3] * qn[3];
        float gq[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) gq[k] = (gqn[k] - qn[k] * qd) / qlen;
        float gls[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) gls[k] = gs[k] * s[k];

        if (out.means) { out.means[3 * i] = gp[0]; out.means[3 * i + 1] = gp[1]; out.means[3 * i + 2] = gp[2]; }
        if (out.log_scales) {
            out.log_scales[3 * i] = gls[0]; out.log_scales[3 * i + 1] = gls[1]; out.log_scales[3 * i + 2] = gls[2];
        }
        if (out.quats) store_n<4>(out.quats + 4 * i, gq);
        if (!sh_stored) {           // several views, or a single view that added nothing (zeros)
            if (out.sh) store_n<K * 3>(out.sh + (long long)K * 3 * i, gH);
            if (out.opacity) {
                if constexpr (VD) store_n<K>(out.opacity + (long long)K * i, gHa);
                else out.opacity[i] = gHa[0];
            }
        }
        if (out.lc_v) out.lc_v[i] = glcv;
    };
    if (det_sb == nullptr) {
        const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        if (i < g.n) body(i);
    } else {
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < g.n;
             i += (long long)gridDim.x * blockDim.x)
            body(i);
    }
    // global weight parameters: warp reduce, then one atomic per warp, or (deterministic) the block's sums
    // in warp order
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        gsig += __shfl_xor_sync(0xffffffffu, gsig, off);
        gbeta += __shfl_xor_sync(0xffffffffu, gbeta, off);
    }
    if (det_sb != nullptr) {
        __shared__ float swb[2][4];
        if ((threadIdx.x & 31) == 0) {
            swb[0][threadIdx.x >> 5] = gsig;
            swb[1][threadIdx.x >> 5] = gbeta;
        }
        __syncthreads();
        if (threadIdx.x < 2) {
            float t = 0.0f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += swb[threadIdx.x][w];
            det_sb[2 * blockIdx.x + threadIdx.x] = t;
        }
    } else if (out.weight_params && wd.kind != WSR_WEIGHT_DIR && (threadIdx.x & 31) == 0) {
        if (gsig != 0.0f) atomicAdd(out.weight_params + 0, gsig);
        if (gbeta != 0.0f) atomicAdd(out.weight_params + 1, gbeta);
    }
}

// Deterministic mode: the blocks' sigma/beta sums added in block order.
__global__ void __launch_bounds__(256) k_det_sb_reduce(const float* __restrict__ sb, int nb, float* __restrict__ gw) {
    __shared__ float part[2][256];
    float a0 = 0.0f, a1 = 0.0f;
    for (int b = threadIdx.x; b < nb; b += 256) {
        a0 += sb[2 * b];
        a1 += sb[2 * b + 1];
    }
    part[0][threadIdx.x] = a0;
    part[1][threadIdx.x] = a1;
    __syncthreads();
    if (threadIdx.x < 2) {
        float t = 0.0f;
        for (int k = 0; k < 256; ++k) t += part[threadIdx.x][k];
        gw[threadIdx.x] = t;
    }
}

template <int DEG, bool VD, bool RED>
cudaError_t project_t(const GaussPtrs& g, const Views& vs, WeightDev w, float* rec, cudaStream_t s) {
    const int bs = 256;
    const long long nb = (g.n + bs - 1) / bs;
    k_project<DEG, VD, RED><<<(unsigned)nb, bs, 0, s>>>(g, vs, w, reinterpret_cast<float4*>(rec));
    return cudaGetLastError();
}

template <int DEG, bool VD, bool RED>
cudaError_t project_bwd_t(const GaussPtrs& g, const Views& vs, WeightDev w, const float* grec,
                          const wsr_grads& out, float* det_sb, cudaStream_t s) {
    const int bs = 128;
    long long nb = (g.n + bs - 1) / bs;
    if (det_sb && nb > kDetSBBlocks) nb = kDetSBBlocks;    // one sigma/beta slot per block
    if (vs.n == 1) k_project_bwd<DEG, VD, RED, true><<<(unsigned)nb, bs, 0, s>>>(g, vs, w, grec, out, det_sb);
    else k_project_bwd<DEG, VD, RED, false><<<(unsigned)nb, bs, 0, s>>>(g, vs, w, grec, out, det_sb);
    if (det_sb) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_det_sb_reduce<<<1, 256, 0, s>>>(det_sb, (int)nb, out.weight_params);
    }
    return cudaGetLastError();
}

template <bool VD, bool RED>
cudaError_t project_deg(const GaussPtrs& g, const Views& vs, WeightDev w, float* rec, cudaStream_t s) {
    switch (g.deg) {
        case 0: return project_t<0, VD, RED>(g, vs, w, rec, s);
        case 1: return project_t<1, VD, RED>(g, vs, w, rec, s);
        case 2: return project_t<2, VD, RED>(g, vs, w, rec, s);
        default: return project_t<3, VD, RED>(g, vs, w, rec, s);
    }
}

template <bool VD, bool RED>
cudaError_t project_bwd_deg(const GaussPtrs& g, const Views& vs, WeightDev w, const float* grec,
                            const wsr_grads& out, float* det_sb, cudaStream_t s) {
    switch (g.deg) {
        case 0: return project_bwd_t<0, VD, RED>(g, vs, w, grec, out, det_sb, s);
        case 1: return project_bwd_t<1, VD, RED>(g, vs, w, grec, out, det_sb, s);
        case 2: return project_bwd_t<2, VD, RED>(g, vs, w, grec, out, det_sb, s);
        default: return project_bwd_t<3, VD, RED>(g, vs, w, grec, out, det_sb, s);
    }
}

}  // namespace

cudaError_t launch_project(const GaussPtrs& g, const Views& vs, WeightDev w, float* rec, cudaStream_t s) {
    if (g.n == 0) return cudaSuccess;
    if (g.vd) return g.red ? project_deg<true, true>(g, vs, w, rec, s) : project_deg<true, false>(g, vs, w, rec, s);
    return g.red ? project_deg<false, true>(g, vs, w, rec, s) : project_deg<false, false>(g, vs, w, rec, s);
}

cudaError_t launch_project_bwd(const GaussPtrs& g, const Views& vs, WeightDev w, const float* grec,
                               const wsr_grads& out, float* det_sb, cudaStream_t s) {
    if (g.n == 0) return cudaSuccess;
    if (g.vd)
        return g.red ? project_bwd_deg<true, true>(g, vs, w, grec, out, det_sb, s)
                     : project_bwd_deg<true, false>(g, vs, w, grec, out, det_sb, s);
    return g.red ? project_bwd_deg<false, true>(g, vs, w, grec, out, det_sb, s)
                 : project_bwd_deg<false, false>(g, vs, w, grec, out, det_sb, s);
}

}  // namespace wsr
