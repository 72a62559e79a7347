/*
 * FP64 reference ("oracle") for Weighted Sum Rendering (WSR), written from
 * "Sort-free Gaussian Splatting via Weighted Sum Rendering" (arXiv 2410.18931).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this file:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg load it.
 * It shares no code, header or constant with the CUDA library.
 *
 * It computes the plain definition, slowly and in double precision:
 *
 *   projection     Sec. 3, Eqs. 3-5 (3D covariance from scale and rotation,
 *                  EWA 2D covariance J W Sigma W^t J^t), 3DGS pre-processing
 *                  kept as Sec. 4.4 / App. A state (0.3 px dilation, Jacobian
 *                  clamp at 1.3 tan(fov), near plane 0.2, 3-sigma footprint).
 *   colour         Eq. 4, real spherical harmonics of degree <= 3 evaluated
 *                  from their closed-form definition (Legendre/Cartesian form,
 *                  Condon-Shortley phase), RGB = max(0, Y.H + 0.5).
 *   opacity        t_i = sigmoid(o_i) (Eq. 3) or the unconstrained
 *                  view-dependent u_i = Y.H^alpha (Eq. 11, not clamped).
 *   weights        Eq. 8 (DIR), Eq. 9 (EXP), Eq. 10 (LC), d_i = camera z.
 *   WSR            Eq. 7: C = (c_B w_B + sum c_i a_i) / (w_B + sum a_i),
 *                  a_i = u_i w(d_i) exp(-q/2), summed over every Gaussian whose
 *                  pixel-centre Mahalanobis distance q <= 9 (3 sigma).
 *   gradient       the analytic derivative of Eq. 7 and of the projection
 *                  chain above with respect to the stored parameters.
 *
 * Readings of points the paper leaves open are listed in the design notes
 * and repeated where they are applied below.
 *
 * Threads: the image renderer splits the image into bands of rows; every pixel
 * still sums its Gaussians in index order, so the result does not depend on
 * the thread count.  The gradient splits the Gaussians; per-Gaussian results
 * are independent and the global sums are added in thread order.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_K 16         /* (deg + 1)^2 for deg <= 3 */
#define ORC_CUTOFF 9.0       /* q <= 9: the 3-sigma footprint */
#define ORC_DILATION 0.3     /* low-pass term added to the 2D covariance */
#define ORC_CLAMP 1.3        /* Jacobian evaluated within 1.3 tan(fov) */

/* Camera as a flat array of 16 doubles: R (row-major 3x3, world -> camera),
 * T (3), fx, fy, cx, cy.  Width, height and the near plane come separately. */
typedef struct {
    double R[9], T[3], fx, fy, cx, cy, znear;
    int W, H;
} ocam;

/* Weight parameters: kind 0 = DIR (Eq. 8), 1 = EXP (Eq. 9), 2 = LC (Eq. 10). */
typedef struct {
    int kind;
    double sigma, beta, w_bg, c_bg[3];
} owt;

typedef struct {
    long n;
    int deg, K, vd;
    const double *means, *log_scales, *quats, *sh, *opac, *lc_v;
} oscene;

/* Everything the projection produces for one Gaussian. */
typedef struct {
    int visible;
    double t[3];          /* camera-space centre */
    double mean2d[2];     /* projected centre, pixels */
    double cov2d[3];      /* Sigma_2D (a, b, c) incl. dilation */
    double conic[3];      /* Sigma_2D^{-1} (A, B, C) */
    double color[3];      /* c_i, after +0.5 and max(0, .) */
    double raw[3];        /* Y.H before the +0.5 offset */
    double u, w, d;       /* opacity, depth weight, depth */
    double dir[3];        /* unit view direction (p - f)/|p - f| */
    double vnorm;         /* |p - f| */
    double rx, ry;        /* 3-sigma half extents along x and y */
    double Y[ORC_MAX_K];  /* SH basis at dir */
} oproj;

static void make_cam(ocam* c, const double* cam16, int W, int H, double znear)
{
    memcpy(c->R, cam16, 9 * sizeof(double));
    memcpy(c->T, cam16 + 9, 3 * sizeof(double));
    c->fx = cam16[12]; c->fy = cam16[13]; c->cx = cam16[14]; c->cy = cam16[15];
    c->W = W; c->H = H; c->znear = znear;
}

static void make_wt(owt* w, int kind, const double* p6)
{
    w->kind = kind;
    w->sigma = p6[0]; w->beta = p6[1]; w->w_bg = p6[2];
    w->c_bg[0] = p6[3]; w->c_bg[1] = p6[4]; w->c_bg[2] = p6[5];
}

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics, degree <= 3 (Eqs. 4 and 11).                     */
/*                                                                            */
/* Closed form on the unit sphere (x, y, z):                                  */
/*   Y_lm = (-1)^m sqrt((2l+1)/(4 pi)) sqrt(2) P_l^|m|(z) A_|m|(x,y)   m > 0  */
/*   Y_lm = (-1)^m sqrt((2l+1)/(4 pi)) sqrt(2) P_l^|m|(z) B_|m|(x,y)   m < 0  */
/*   Y_l0 = sqrt((2l+1)/(4 pi)) P_l^0(z)                                      */
/* with                                                                       */
/*   P_l^m(z) = sqrt((l-m)!/(l+m)!) sum_k (-1)^k 2^-l C(l,k) C(2l-2k,l)       */
/*              (l-2k)!/(l-2k-m)! z^(l-2k-m)          (k <= (l-m)/2, r = 1)   */
/*   A_m = sum_p C(m,p) x^p y^(m-p) cos((m-p) pi/2)                           */
/*   B_m = sum_p C(m,p) x^p y^(m-p) sin((m-p) pi/2)                           */
/* Index of (l, m) is l^2 + l + m.  The (-1)^m factor is the Condon-Shortley  */
/* phase.  The gradient is that of the polynomial in (x, y, z); callers take  */
/* its tangential part, which is all that matters on the sphere.              */
/* ------------------------------------------------------------------------ */
static double fact(int n) { double r = 1; for (int i = 2; i <= n; ++i) r *= i; return r; }
static double binom(int n, int k) { return fact(n) / (fact(k) * fact(n - k)); }
static double ipow(double x, int n) { double r = 1; for (int i = 0; i < n; ++i) r *= x; return r; }
static double dipow(double x, int n) { return n == 0 ? 0.0 : n * ipow(x, n - 1); }

static void sh_basis(int deg, const double d[3], double* Y, double (*dY)[3])
{
    const double x = d[0], y = d[1], z = d[2];
    for (int l = 0; l <= deg; ++l) {
        const double Kl = sqrt((2.0 * l + 1.0) / (4.0 * M_PI));
        for (int m = -l; m <= l; ++m) {
            const int am = m < 0 ? -m : m;
            /* associated Legendre part P_l^am(z) and its z-derivative */
            double P = 0, dP = 0;
            for (int k = 0; 2 * k <= l - am; ++k) {
                const double c = ipow(-1.0, k) * ldexp(1.0, -l) * binom(l, k) *
                                 binom(2 * l - 2 * k, l) * fact(l - 2 * k) / fact(l - 2 * k - am);
                P += c * ipow(z, l - 2 * k - am);
                dP += c * dipow(z, l - 2 * k - am);
            }
            const double norm = sqrt(fact(l - am) / fact(l + am));
            P *= norm; dP *= norm;
            /* azimuthal part */
            double S = 1, dSx = 0, dSy = 0, pref = Kl;
            if (m != 0) {
                S = 0;
                for (int p = 0; p <= am; ++p) {
                    const double ang = (am - p) * M_PI / 2.0;
                    /* cos / sin of multiples of pi/2 are exactly 0, +-1 */
                    const double tr = (m > 0) ? (double)lround(cos(ang)) : (double)lround(sin(ang));
                    const double c = binom(am, p) * tr;
                    S += c * ipow(x, p) * ipow(y, am - p);
                    dSx += c * dipow(x, p) * ipow(y, am - p);
                    dSy += c * ipow(x, p) * dipow(y, am - p);
                }
                pref = Kl * sqrt(2.0) * ipow(-1.0, am);
            }
            const int idx = l * l + l + m;
            Y[idx] = pref * P * S;
            if (dY) {
                dY[idx][0] = pref * P * dSx;
                dY[idx][1] = pref * P * dSy;
                dY[idx][2] = pref * dP * S;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Small dense helpers (row-major).                                          */
/* ------------------------------------------------------------------------ */
static void mat_mul(const double* A, const double* B, double* C, int n, int k, int m)
{   /* C[n x m] = A[n x k] B[k x m] */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) {
            double s = 0;
            for (int t = 0; t < k; ++t) s += A[i * k + t] * B[t * m + j];
            C[i * m + j] = s;
        }
}
static void transpose(const double* A, double* At, int n, int m)
{   /* At[m x n] = A[n x m]^t */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) At[j * n + i] = A[i * m + j];
}

/* Rotation matrix of the unit quaternion (w, x, y, z) (Hamilton convention). */
static void quat_to_rot(const double q[4], double R[9])
{
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}
/* dR[e][c]: derivative of R entry e with respect to quaternion component c. */
static void quat_to_rot_grad(const double q[4], double dR[9][4])
{
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    const double g[9][4] = {
        {0, 0, -4 * y, -4 * z},   {-2 * z, 2 * y, 2 * x, -2 * w}, {2 * y, 2 * z, 2 * w, 2 * x},
        {2 * z, 2 * y, 2 * x, 2 * w}, {0, -4 * x, 0, -4 * z},     {-2 * x, -2 * w, 2 * z, 2 * y},
        {-2 * y, 2 * z, -2 * w, 2 * x}, {2 * x, 2 * w, 2 * z, 2 * y}, {0, -4 * x, -4 * y, 0}};
    memcpy(dR, g, sizeof g);
}

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* ------------------------------------------------------------------------ */
/* Projection of one Gaussian (Sec. 3, Eqs. 3-5, 4, 11, 8-10).              */
/* ------------------------------------------------------------------------ */
static void project_one(const oscene* S, long i, const ocam* cam, const owt* wt, oproj* o)
{
    memset(o, 0, sizeof *o);
    const double* p = S->means + 3 * i;
    /* camera space t = W p + T */
    for (int r = 0; r < 3; ++r)
        o->t[r] = cam->R[3 * r] * p[0] + cam->R[3 * r + 1] * p[1] + cam->R[3 * r + 2] * p[2] + cam->T[r];
    o->d = o->t[2];
    if (!(o->t[2] > cam->znear)) { o->visible = 0; return; }   /* near-plane cull (App. C) */
    o->visible = 1;
    const double tx = o->t[0], ty = o->t[1], tz = o->t[2];

    /* Sigma_3D = R S S^t R^t (Eq. 3) */
    const double* qr = S->quats + 4 * i;
    const double qn = sqrt(qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3]);
    const double q[4] = {qr[0] / qn, qr[1] / qn, qr[2] / qn, qr[3] / qn};
    double Rg[9], M[9], Mt[9], Sig3[9];
    quat_to_rot(q, Rg);
    double s[3];
    for (int k = 0; k < 3; ++k) s[k] = exp(S->log_scales[3 * i + k]);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) M[3 * r + c] = Rg[3 * r + c] * s[c];   /* M = R S */
    transpose(M, Mt, 3, 3);
    mat_mul(M, Mt, Sig3, 3, 3, 3);

    /* Sigma_2D = J W Sigma_3D W^t J^t + 0.3 I (Eq. 5) */
    const double tanx = 0.5 * cam->W / cam->fx, tany = 0.5 * cam->H / cam->fy;
    const double rxc = clampd(tx / tz, -ORC_CLAMP * tanx, ORC_CLAMP * tanx);
    const double ryc = clampd(ty / tz, -ORC_CLAMP * tany, ORC_CLAMP * tany);
    const double J[6] = {cam->fx / tz, 0, -cam->fx * rxc / tz, 0, cam->fy / tz, -cam->fy * ryc / tz};
    double JW[6], JWt[6], tmp[6], S2[4];
    mat_mul(J, cam->R, JW, 2, 3, 3);
    mat_mul(JW, Sig3, tmp, 2, 3, 3);
    transpose(JW, JWt, 2, 3);
    mat_mul(tmp, JWt, S2, 2, 3, 2);
    const double a = S2[0] + ORC_DILATION, b = 0.5 * (S2[1] + S2[2]), c = S2[3] + ORC_DILATION;
    o->cov2d[0] = a; o->cov2d[1] = b; o->cov2d[2] = c;
    const double det = a * c - b * b;
    o->conic[0] = c / det; o->conic[1] = -b / det; o->conic[2] = a / det;
    o->mean2d[0] = cam->fx * tx / tz + cam->cx;
    o->mean2d[1] = cam->fy * ty / tz + cam->cy;
    o->rx = 3.0 * sqrt(a);
    o->ry = 3.0 * sqrt(c);

    /* view direction from the camera centre f = -R^t T to the Gaussian */
    double f[3], v[3];
    for (int k = 0; k < 3; ++k)
        f[k] = -(cam->R[k] * cam->T[0] + cam->R[3 + k] * cam->T[1] + cam->R[6 + k] * cam->T[2]);
    for (int k = 0; k < 3; ++k) v[k] = p[k] - f[k];
    o->vnorm = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int k = 0; k < 3; ++k) o->dir[k] = v[k] / o->vnorm;
    sh_basis(S->deg, o->dir, o->Y, NULL);

    /* colour (Eq. 4) */
    const double* H = S->sh + (long)i * S->K * 3;
    for (int ch = 0; ch < 3; ++ch) {
        double r = 0;
        for (int k = 0; k < S->K; ++k) r += o->Y[k] * H[3 * k + ch];
        o->raw[ch] = r;
        o->color[ch] = r + 0.5 > 0 ? r + 0.5 : 0.0;
    }
    /* opacity: view-dependent (Eq. 11, unclamped) or sigmoid of a logit */
    if (S->vd) {
        const double* Ha = S->opac + (long)i * S->K;
        double u = 0;
        for (int k = 0; k < S->K; ++k) u += o->Y[k] * Ha[k];
        o->u = u;
    } else {
        o->u = 1.0 / (1.0 + exp(-S->opac[i]));
    }
    /* depth weight (Eqs. 8-10) */
    const double d = o->d;
    if (wt->kind == 0) o->w = 1.0;
    else if (wt->kind == 1) o->w = exp(-wt->sigma * pow(d, wt->beta));
    else {
        const double lin = 1.0 - d / wt->sigma;
        o->w = (lin > 0 ? lin : 0.0) * S->lc_v[i];
    }
}

/* Pixel-index range whose centres can fall within the footprint (with one
 * pixel of slack; the q test decides). */
static void pixel_range(const oproj* o, const ocam* cam, double grow, int* x0, int* x1, int* y0, int* y1)
{
    const double rx = o->rx * grow, ry = o->ry * grow;
    *x0 = (int)floor(o->mean2d[0] - rx - 0.5) - 1;
    *x1 = (int)ceil(o->mean2d[0] + rx - 0.5) + 1;
    *y0 = (int)floor(o->mean2d[1] - ry - 0.5) - 1;
    *y1 = (int)ceil(o->mean2d[1] + ry - 0.5) + 1;
    if (*x0 < 0) *x0 = 0;
    if (*y0 < 0) *y0 = 0;
    if (*x1 > cam->W - 1) *x1 = cam->W - 1;
    if (*y1 > cam->H - 1) *y1 = cam->H - 1;
}

static double quad_form(const double conic[3], double dx, double dy)
{
    return conic[0] * dx * dx + 2.0 * conic[1] * dx * dy + conic[2] * dy * dy;
}

/* ------------------------------------------------------------------------ */
/* Cutoff ties: how far an FP32 renderer's q can lie from q.                 */
/*                                                                          */
/* Eq. 7 sums the pairs with q <= 9.  A renderer that works in FP32 decides  */
/* that test from a record rounded to FP32 (the projected mean, and the     */
/* conic held as the sum of squares q = (qs dy + qw dx)^2 + qd dx^2 of      */
/* Sigma_2D = T T^t + 0.3 I, T = J W R S formed in FP32), so a pair whose q */
/* lies within that rounding of 9 may be decided the other way there.  The  */
/* comparison of such a renderer with this oracle forgives exactly those    */
/* pairs; tie_width() bounds |q_FP32 - q| for one pair, to first order in   */
/* the FP32 unit roundoff u = 2^-24 (IEEE operations; exp within 2 ulp),    */
/* term by term (v = Sigma^-1 d, d the pixel's offset from the mean):       */
/*   mean    2 (|v_x| e_x + |v_y| e_y), e the bound on the FP32 mean's      */
/*           error: t = W p + T, then fx t_x / t_z + c_x;                   */
/*   rows    2 |T^t v| |(|dT|^t |v|)|, dT the bound on the FP32 error of    */
/*           each entry of T (from R of the normalised quaternion, exp of   */
/*           the log-scales, W R S, and J at the FP32 t);                    */
/*   sums    |v|^t E |v|, E the rounding of a, b, c from the rows, the FP32 */
/*           constant 0.3, and the determinant |r0 x r1|^2 + 0.3 (a0 + c0)  */
/*           + 0.09 rounded (an error in it acts as one in c); none of it   */
/*           when the conic is formed in FP64 (det < 1e-3 a c);             */
/*   record  the rounding of qd, qs and qw themselves;                      */
/*   test    evaluating q at the pixel (any order of a dozen FMAs, offsets  */
/*           of up to 62 pixels from a tile origin) and the FP32 threshold; */
/* and doubles the sum for the second-order terms.  It is test              */
/* infrastructure: no part of Eq. 7 depends on it.                          */
/* ------------------------------------------------------------------------ */
#define ORC_U (1.0 / 16777216.0)    /* FP32 unit roundoff, 2^-24 */
/* Widest tie window the pixel ranges cover: they reach q = 9 + ORC_TIE_CAP.
 * Every term of the window grows at most linearly in q, so if each pair
 * within ORC_TIE_CAP of the cutoff has a window under ORC_TIE_CAP / 2, no pair
 * beyond the ranges (q > 9 + ORC_TIE_CAP) can be a tie; callers report a
 * window that breaks this (too_wide). */
#define ORC_TIE_CAP 1.0

static double gam(int n) { return n * ORC_U / (1.0 - n * ORC_U); }

typedef struct {
    double ex, ey;          /* bound on the FP32 mean's error (pixels) */
    double T[6], eT[6];     /* rows of T = J W R S, and bounds on their FP32 errors */
    double E[3];            /* rounding of Sigma's a, b, c (the determinant's folded into c) */
    double eta_d, eta_s, eta_w;  /* relative rounding of qd, qs, qw */
    double qs, qw, qd;      /* Sigma^-1 as the sum of squares (q units) */
} otie;

static void tie_model(const oscene* S, long i, const ocam* cam, const oproj* o, otie* m)
{
    const double u = ORC_U;
    memset(m, 0, sizeof *m);
    if (!o->visible) return;
    const double* p = S->means + 3 * i;
    /* t = W p + T: three products, three sums per entry */
    double et[3];
    for (int r = 0; r < 3; ++r)
        et[r] = gam(4) * (fabs(cam->R[3 * r] * p[0]) + fabs(cam->R[3 * r + 1] * p[1]) +
                          fabs(cam->R[3 * r + 2] * p[2]) + fabs(cam->T[r]));
    const double tz = o->t[2], ux = o->t[0] / tz, uy = o->t[1] / tz;
    /* mean fx t_x / t_z + c_x: the error of t, then a product, a quotient and a sum */
    m->ex = cam->fx * (et[0] + fabs(ux) * et[2]) / tz + 2 * u * cam->fx * fabs(ux) + u * fabs(o->mean2d[0]);
    m->ey = cam->fy * (et[1] + fabs(uy) * et[2]) / tz + 2 * u * cam->fy * fabs(uy) + u * fabs(o->mean2d[1]);
    /* R of the normalised quaternion: every entry within 32 u (|q| = 1 and a few roundings
     * each); exp within 2 ulp (4 u); M = W R S with its 3-term sums */
    const double* qr = S->quats + 4 * i;
    const double ql = sqrt(qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3]);
    const double qu[4] = {qr[0] / ql, qr[1] / ql, qr[2] / ql, qr[3] / ql};
    double Rq[9], M[9], eM[9], sc[3];
    quat_to_rot(qu, Rq);
    for (int k = 0; k < 3; ++k) sc[k] = exp(S->log_scales[3 * i + k]);
    for (int r = 0; r < 3; ++r)
        for (int cc = 0; cc < 3; ++cc) {
            double v = 0, av = 0, aw = 0;
            for (int k = 0; k < 3; ++k) {
                v += cam->R[3 * r + k] * Rq[3 * k + cc];
                av += fabs(cam->R[3 * r + k] * Rq[3 * k + cc]);
                aw += fabs(cam->R[3 * r + k]);
            }
            M[3 * r + cc] = v * sc[cc];
            eM[3 * r + cc] = sc[cc] * (gam(3) * av + 32 * u * aw) + 5 * u * fabs(M[3 * r + cc]);
        }
    /* J at the clamped x/z, y/z of the FP32 t; the FP32 clamp limit differs by u */
    const double eiz = u + et[2] / tz;
    const double limx = ORC_CLAMP * 0.5 * cam->W / cam->fx, limy = ORC_CLAMP * 0.5 * cam->H / cam->fy;
    const double cxz = clampd(ux, -limx, limx), cyz = clampd(uy, -limy, limy);
    const double ecx = et[0] / tz + fabs(ux) * (eiz + u) + u * limx;
    const double ecy = et[1] / tz + fabs(uy) * (eiz + u) + u * limy;
    const double J00 = cam->fx / tz, J02 = -cam->fx * cxz / tz, J11 = cam->fy / tz, J12 = -cam->fy * cyz / tz;
    const double eJ00 = J00 * (eiz + u), eJ11 = J11 * (eiz + u);
    const double eJ02 = cam->fx / tz * (ecx + fabs(cxz) * (eiz + 2 * u));
    const double eJ12 = cam->fy / tz * (ecy + fabs(cyz) * (eiz + 2 * u));
    for (int k = 0; k < 3; ++k) {
        m->T[k] = J00 * M[k] + J02 * M[6 + k];
        m->T[3 + k] = J11 * M[3 + k] + J12 * M[6 + k];
        m->eT[k] = eJ00 * fabs(M[k]) + J00 * eM[k] + eJ02 * fabs(M[6 + k]) + fabs(J02) * eM[6 + k] +
                   gam(2) * (fabs(J00 * M[k]) + fabs(J02 * M[6 + k]));
        m->eT[3 + k] = eJ11 * fabs(M[3 + k]) + J11 * eM[3 + k] + eJ12 * fabs(M[6 + k]) + fabs(J12) * eM[6 + k] +
                       gam(2) * (fabs(J11 * M[3 + k]) + fabs(J12 * M[6 + k]));
    }
    const double a = o->cov2d[0], b = o->cov2d[1], c = o->cov2d[2], det = a * c - b * b;
    m->qd = 1.0 / a;
    m->qs = sqrt(a / det);
    m->qw = -(b / a) * m->qs;
    if (det < 0.999e-3 * a * c) {
        /* formed in FP64 from the FP32 rows: only the final rounding of qd, qs, qw */
        m->eta_d = m->eta_s = m->eta_w = u;
        return;
    }
    const double* r0 = m->T;
    const double* r1 = m->T + 3;
    double a0 = 0, c0 = 0, babs = 0, x2 = 0, edet = 0;
    for (int k = 0; k < 3; ++k) {
        a0 += r0[k] * r0[k];
        c0 += r1[k] * r1[k];
        babs += fabs(r0[k] * r1[k]);
        const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
        const double x = r0[k1] * r1[k2] - r0[k2] * r1[k1];
        x2 += x * x;
        edet += 2 * fabs(x) * gam(2) * (fabs(r0[k1] * r1[k2]) + fabs(r0[k2] * r1[k1]));
    }
    const double d03 = fabs(0.3 - (double)0.3f);
    const double ea = gam(3) * a0 + u * a, eb = gam(3) * babs;
    edet += gam(3) * x2 + 2 * u * 0.3 * (a0 + c0) + u * 0.09 + 2 * u * det;
    m->E[0] = ea + d03;
    m->E[1] = eb;
    m->E[2] = gam(3) * c0 + u * c + d03 + (edet + 2 * fabs(b) * eb + c * ea) / a;
    m->eta_d = 2 * u;
    m->eta_s = 3 * u;
    m->eta_w = 2 * u;
}

/* The tie window of one pair (pixel offset dx, dy from the mean; q its exact
 * value); terms[6], if given, gets its six parts (mean, rows, sums, record,
 * threshold, evaluation), each doubled as in the window. */
static double tie_width(const otie* m, double dx, double dy, double q, double* terms)
{
    const double u = ORC_U;
    const double r = m->qs * dy + m->qw * dx;
    const double vx = m->qw * r + m->qd * dx, vy = m->qs * r;     /* v = Sigma^-1 d = grad(q) / 2 */
    const double t_mean = 2.0 * (fabs(vx) * m->ex + fabs(vy) * m->ey);
    double tv2 = 0, ev2 = 0;
    for (int k = 0; k < 3; ++k) {
        const double tk = m->T[k] * vx + m->T[3 + k] * vy;
        const double ek = m->eT[k] * fabs(vx) + m->eT[3 + k] * fabs(vy);
        tv2 += tk * tk;
        ev2 += ek * ek;
    }
    const double t_rows = 2.0 * sqrt(tv2 * ev2);
    const double t_sums = m->E[0] * vx * vx + 2 * m->E[1] * fabs(vx * vy) + m->E[2] * vy * vy;
    const double t_rec = 2 * m->eta_s * r * r + 2 * m->eta_w * fabs(r * m->qw * dx) + m->eta_d * m->qd * dx * dx;
    const double t_cut = 18 * u;                 /* 9 k with k = log2(e) / 2, each rounded to FP32 */
    const double X = fabs(dx) + 62.0, Y = fabs(dy) + 62.0;
    const double t_eval = 12 * u * fabs(r) * (m->qs * Y + fabs(m->qw) * X) + 6 * u * m->qd * X * X + u * q;
    if (terms) {
        terms[0] = 2.0 * t_mean;
        terms[1] = 2.0 * t_rows;
        terms[2] = 2.0 * t_sums;
        terms[3] = 2.0 * t_rec;
        terms[4] = 2.0 * t_cut;
        terms[5] = 2.0 * t_eval;
    }
    return 2.0 * (t_mean + t_rows + t_sums + t_rec + t_cut + t_eval);
}

/* Test hook: with a nonzero seed, a pair within orc_flip_tau of the cutoff is
 * counted or not by a hash of (seed, Gaussian, pixel) instead of q <= 9, in
 * the forward sums (which = 0) or in the gradient's sums (which = 1).  It
 * stands in for a renderer that decides ties either way, so that tests can
 * check the tie bounds against arbitrary decisions. */
static unsigned orc_flip_seed[2];
static double orc_flip_tau;

void wsro_set_tie_flips(unsigned fwd_seed, unsigned grad_seed, double tau)
{
    orc_flip_seed[0] = fwd_seed;
    orc_flip_seed[1] = grad_seed;
    orc_flip_tau = tau;
}

static int counted(double q, double cutoff, long i, int x, int y, int which)
{
    const unsigned seed = orc_flip_seed[which];
    if (seed && fabs(q - ORC_CUTOFF) <= orc_flip_tau) {
        uint64_t h = ((uint64_t)seed << 32) ^ ((uint64_t)i * 0x9E3779B97F4A7C15ull) ^
                     ((uint64_t)(unsigned)x << 20) ^ (uint64_t)(unsigned)y;
        h ^= h >> 33; h *= 0xFF51AFD7ED558CCDull; h ^= h >> 33; h *= 0xC4CEB9FE1A85EC53ull; h ^= h >> 33;
        return (int)(h & 1u);
    }
    return q <= cutoff;
}

static int too_wide(double q, double tau) { return fabs(q - ORC_CUTOFF) <= ORC_TIE_CAP && tau > 0.5 * ORC_TIE_CAP; }

/* Models of every Gaussian (malloc'ed). */
static otie* tie_all(const oscene* S, const ocam* cam, const oproj* P)
{
    otie* m = (otie*)malloc(sizeof(otie) * (S->n > 0 ? S->n : 1));
    if (!m) return NULL;
    for (long i = 0; i < S->n; ++i) tie_model(S, i, cam, P + i, m + i);
    return m;
}

/* ------------------------------------------------------------------------ */
/* Thread helper                                                             */
/* ------------------------------------------------------------------------ */
typedef struct { void (*fn)(void*, long, long, int); void* arg; long lo, hi; int tid; } ojob;
static void* job_main(void* p) { ojob* j = (ojob*)p; j->fn(j->arg, j->lo, j->hi, j->tid); return NULL; }
static void run_parallel(void (*fn)(void*, long, long, int), void* arg, long n, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (nthreads == 1 || n < 2) { fn(arg, 0, n, 0); return; }
    pthread_t th[256];
    ojob jobs[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].fn = fn; jobs[t].arg = arg; jobs[t].tid = t;
        jobs[t].lo = n * t / nthreads; jobs[t].hi = n * (t + 1) / nthreads;
        pthread_create(&th[t], NULL, job_main, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
}

static void fill_scene(oscene* S, long n, int deg, int vd, const double* means, const double* log_scales,
                       const double* quats, const double* sh, const double* opac, const double* lc_v)
{
    S->n = n; S->deg = deg; S->K = (deg + 1) * (deg + 1); S->vd = vd;
    S->means = means; S->log_scales = log_scales; S->quats = quats; S->sh = sh;
    S->opac = opac; S->lc_v = lc_v;
}

/* ------------------------------------------------------------------------ */
/* Public: projection table                                                  */
/* out[n][ORC_PROJ_STRIDE]: visible, t(3), mean2d(2), cov2d(3), conic(3),     */
/* color(3), u, w, d, rx, ry                                                  */
/* ------------------------------------------------------------------------ */
#define ORC_PROJ_STRIDE 22
int wsro_project(long n, int deg, int vd, const double* means, const double* log_scales,
                 const double* quats, const double* sh, const double* opac, const double* lc_v,
                 const double* cam16, int W, int H, double znear, int wkind, const double* wpar,
                 double* out)
{
    if (deg < 0 || deg > 3 || n < 0) return 1;
    oscene S; ocam cam; owt wt;
    fill_scene(&S, n, deg, vd, means, log_scales, quats, sh, opac, lc_v);
    make_cam(&cam, cam16, W, H, znear);
    make_wt(&wt, wkind, wpar);
    for (long i = 0; i < n; ++i) {
        oproj o;
        project_one(&S, i, &cam, &wt, &o);
        double* r = out + i * ORC_PROJ_STRIDE;
        r[0] = o.visible;
        memcpy(r + 1, o.t, 3 * sizeof(double));
        memcpy(r + 4, o.mean2d, 2 * sizeof(double));
        memcpy(r + 6, o.cov2d, 3 * sizeof(double));
        memcpy(r + 9, o.conic, 3 * sizeof(double));
        memcpy(r + 12, o.color, 3 * sizeof(double));
        r[15] = o.u; r[16] = o.w; r[17] = o.d; r[18] = o.rx; r[19] = o.ry;
        r[20] = 0; r[21] = 0;
    }
    return 0;
}

/* Real SH basis (and its polynomial gradient) at unit directions. */
int wsro_sh_basis(long n, int deg, const double* dirs, double* Y /* n x K */, double* dY /* n x K x 3 or NULL */)
{
    if (deg < 0 || deg > 3) return 1;
    const int K = (deg + 1) * (deg + 1);
    for (long i = 0; i < n; ++i) {
        double y[ORC_MAX_K], dy[ORC_MAX_K][3];
        sh_basis(deg, dirs + 3 * i, y, dy);
        memcpy(Y + i * K, y, K * sizeof(double));
        if (dY) memcpy(dY + i * K * 3, dy, K * 3 * sizeof(double));
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Public: full-image forward (Eq. 7)                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    const oproj* P; long n; const ocam* cam; const owt* wt;
    double cutoff;           /* footprint test q <= cutoff (9 for Eq. 7 as read here) */
    int y_lo;                /* first image row of the window held in the buffers */
    double *num, *den;       /* [rows*W*3], [rows*W] sums (without background) */
    long long* pairs;        /* per thread */
    double amb_tau;          /* window around the cutoff */
    double* amb;             /* [H*W] or NULL: filled in a second pass */
    const double* rgb;       /* final colours, for the second pass */
    const double* dent;      /* total denominators, for the second pass */
    const otie* tie;         /* per-pair windows from the FP32 model (NULL: amb_tau for every pair) */
    double* mass;            /* [H*W] or NULL: sum of |a| over the pixel's tie pairs */
    int* wide;               /* per thread: a model window broke the ORC_TIE_CAP rule (too_wide) */
} render_ctx;

static void render_rows(void* arg, long r0, long r1, int tid)
{
    render_ctx* c = (render_ctx*)arg;
    r0 += c->y_lo;
    r1 += c->y_lo;
    const int W = c->cam->W;
    long long pairs = 0;
    const double widest = c->amb ? (c->tie ? ORC_TIE_CAP : c->amb_tau) : 0.0;
    const double grow = sqrt((c->cutoff + widest + (orc_flip_seed[0] ? orc_flip_tau : 0.0)) / ORC_CUTOFF);
    for (long i = 0; i < c->n; ++i) {
        const oproj* o = c->P + i;
        if (!o->visible) continue;
        int x0, x1, y0, y1;
        pixel_range(o, c->cam, grow, &x0, &x1, &y0, &y1);
        if (y0 < r0) y0 = (int)r0;
        if (y1 > r1 - 1) y1 = (int)(r1 - 1);
        for (int y = y0; y <= y1; ++y)
            for (int x = x0; x <= x1; ++x) {
                const double dx = x + 0.5 - o->mean2d[0], dy = y + 0.5 - o->mean2d[1];
                const double q = quad_form(o->conic, dx, dy);
                const long p = (long)(y - c->y_lo) * W + x;
                if (c->amb) {
                    /* second pass: bound of what a near-cutoff pair can change */
                    const double tau = c->tie ? tie_width(c->tie + i, dx, dy, q, NULL) : c->amb_tau;
                    if (c->tie ? too_wide(q, tau) : tau > widest) c->wide[tid] = 1;
                    if (fabs(q - c->cutoff) <= tau) {
                        const double g = exp(-0.5 * q);
                        const double a = o->u * o->w * g;
                        double m = 0;
                        for (int ch = 0; ch < 3; ++ch) {
                            const double e = fabs(o->color[ch] - c->rgb[3 * p + ch]);
                            if (e > m) m = e;
                        }
                        c->amb[p] += fabs(a) * m;          /* divided by the least |D| afterwards */
                        c->mass[p] += fabs(a);
                    }
                    continue;
                }
                if (!counted(q, c->cutoff, i, x, y, 0)) continue;
                const double g = exp(-0.5 * q);
                const double a = o->u * o->w * g;            /* alpha_i w(d_i) */
                for (int ch = 0; ch < 3; ++ch) c->num[3 * p + ch] += o->color[ch] * a;
                c->den[p] += a;
                ++pairs;
            }
    }
    c->pairs[tid] = pairs;
}

/* Project every Gaussian once (index order). Returns malloc'ed table. */
static oproj* project_all(const oscene* S, const ocam* cam, const owt* wt)
{
    oproj* P = (oproj*)malloc(sizeof(oproj) * (S->n > 0 ? S->n : 1));
    if (!P) return NULL;
    for (long i = 0; i < S->n; ++i) project_one(S, i, cam, wt, P + i);
    return P;
}

/*
 * Rows [y_lo, y_hi) of the image (the whole image for 0, H).  `cutoff` is the
 * footprint bound on q (9: the 3-sigma footprint); other values serve tests
 * that bracket pairs whose q is within rounding of 9.
 * out_rgb [rows*W*3]: C per pixel (Eq. 7); out_den [rows*W]: w_B + sum a_i.
 * amb [H*W] (optional): for pixels having Gaussians with |q - 9| <= amb_tau,
 * a bound on how far C can move if those pairs were decided the other way;
 * amb_tau < 0 takes each pair's window from the FP32 rounding model above.
 * tie_mass [H*W] (optional, with amb): the sum of |a| over those pairs.
 * n_pairs (optional): number of (pixel, Gaussian) pairs with q <= 9.
 * Returns 3 if a model window broke the ORC_TIE_CAP rule (the pixel ranges would
 * then miss pairs).
 */
int wsro_render(long n, int deg, int vd, const double* means, const double* log_scales,
                const double* quats, const double* sh, const double* opac, const double* lc_v,
                const double* cam16, int W, int H, double znear, int wkind, const double* wpar,
                int nthreads, int y_lo, int y_hi, double* out_rgb, double* out_den, double* amb,
                double amb_tau, long long* n_pairs, double cutoff, double* tie_mass)
{
    if (deg < 0 || deg > 3 || n < 0 || W <= 0 || H <= 0) return 1;
    if (y_lo < 0 || y_hi > H || y_lo >= y_hi) return 1;
    const int rows = y_hi - y_lo;
    oscene S; ocam cam; owt wt;
    fill_scene(&S, n, deg, vd, means, log_scales, quats, sh, opac, lc_v);
    make_cam(&cam, cam16, W, H, znear);
    make_wt(&wt, wkind, wpar);
    oproj* P = project_all(&S, &cam, &wt);
    if (!P) return 2;
    const long np = (long)W * rows;
    double* num = (double*)calloc(np * 3, sizeof(double));
    double* den = (double*)calloc(np, sizeof(double));
    long long pairs[256] = {0};
    render_ctx c = {P, n, &cam, &wt, cutoff, y_lo, num, den, pairs, amb_tau, NULL, NULL, NULL, NULL, NULL, NULL};
    if (nthreads > rows) nthreads = rows;
    run_parallel(render_rows, &c, rows, nthreads);
    long long tot = 0;
    for (int t = 0; t < 256; ++t) tot += pairs[t];
    if (n_pairs) *n_pairs = tot;
    for (long p = 0; p < np; ++p) {
        const double D = wt.w_bg + den[p];
        out_den[p] = D;
        for (int ch = 0; ch < 3; ++ch) out_rgb[3 * p + ch] = (wt.c_bg[ch] * wt.w_bg + num[3 * p + ch]) / D;
    }
    int rc = 0;
    if (amb) {
        /* a pixel's tie pairs move C by sum |a| |c - C| / |D'| at most, D' the denominator
         * after the other decisions: |D'| >= |D| - sum |a| (infinite if D' can vanish) */
        double* mass = tie_mass ? tie_mass : (double*)malloc(np * sizeof(double));
        otie* tm = amb_tau < 0 ? tie_all(&S, &cam, P) : NULL;
        int wide[256] = {0};
        if (!mass || (amb_tau < 0 && !tm)) {
            rc = 2;
        } else {
            memset(amb, 0, np * sizeof(double));
            memset(mass, 0, np * sizeof(double));
            render_ctx c2 = {P, n, &cam, &wt, cutoff, y_lo, NULL, NULL, pairs, amb_tau, amb, out_rgb, out_den,
                             tm, mass, wide};
            run_parallel(render_rows, &c2, rows, nthreads);
            for (long p = 0; p < np; ++p) {
                const double dlo = fabs(out_den[p]) - mass[p];
                if (amb[p] > 0) amb[p] = dlo > 0 ? amb[p] / dlo : HUGE_VAL;
            }
            for (int t = 0; t < 256; ++t) if (wide[t]) rc = 3;
        }
        if (!tie_mass) free(mass);
        free(tm);
    }
    free(num); free(den); free(P);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Public: forward at a list of pixels, each summed over all Gaussians.      */
/* ------------------------------------------------------------------------ */
typedef struct {
    const oproj* P; long n; const ocam* cam; const owt* wt;
    const int* xy; double *rgb, *den, *amb; double amb_tau;
} pix_ctx;

static void render_pixels(void* arg, long lo, long hi, int tid)
{
    (void)tid;
    pix_ctx* c = (pix_ctx*)arg;
    for (long k = lo; k < hi; ++k) {
        const int x = c->xy[2 * k], y = c->xy[2 * k + 1];
        double num[3] = {0, 0, 0}, den = 0;
        for (long i = 0; i < c->n; ++i) {
            const oproj* o = c->P + i;
            if (!o->visible) continue;
            const double dx = x + 0.5 - o->mean2d[0], dy = y + 0.5 - o->mean2d[1];
            if (fabs(dx) > o->rx + 1.0 || fabs(dy) > o->ry + 1.0) continue;
            const double q = quad_form(o->conic, dx, dy);
            if (q > ORC_CUTOFF) continue;
            const double a = o->u * o->w * exp(-0.5 * q);
            for (int ch = 0; ch < 3; ++ch) num[ch] += o->color[ch] * a;
            den += a;
        }
        const double D = c->wt->w_bg + den;
        double C[3];
        for (int ch = 0; ch < 3; ++ch) C[ch] = (c->wt->c_bg[ch] * c->wt->w_bg + num[ch]) / D;
        double am = 0, mass = 0;
        if (c->amb) {
            const double grow = sqrt((ORC_CUTOFF + c->amb_tau) / ORC_CUTOFF);
            for (long i = 0; i < c->n; ++i) {
                const oproj* o = c->P + i;
                if (!o->visible) continue;
                const double dx = x + 0.5 - o->mean2d[0], dy = y + 0.5 - o->mean2d[1];
                if (fabs(dx) > o->rx * grow + 1.0 || fabs(dy) > o->ry * grow + 1.0) continue;
                const double q = quad_form(o->conic, dx, dy);
                if (fabs(q - ORC_CUTOFF) > c->amb_tau) continue;
                const double a = o->u * o->w * exp(-0.5 * q);
                double m = 0;
                for (int ch = 0; ch < 3; ++ch) { const double e = fabs(o->color[ch] - C[ch]); if (e > m) m = e; }
                am += fabs(a) * m;
                mass += fabs(a);
            }
            /* divided by the least |D| the tie decisions allow */
            c->amb[k] = am > 0 ? (fabs(D) > mass ? am / (fabs(D) - mass) : HUGE_VAL) : 0.0;
        }
        for (int ch = 0; ch < 3; ++ch) c->rgb[3 * k + ch] = C[ch];
        c->den[k] = D;
    }
}

int wsro_render_pixels(long n, int deg, int vd, const double* means, const double* log_scales,
                       const double* quats, const double* sh, const double* opac, const double* lc_v,
                       const double* cam16, int W, int H, double znear, int wkind, const double* wpar,
                       int nthreads, long npix, const int* xy, double* out_rgb, double* out_den,
                       double* amb, double amb_tau)
{
    if (deg < 0 || deg > 3 || n < 0) return 1;
    oscene S; ocam cam; owt wt;
    fill_scene(&S, n, deg, vd, means, log_scales, quats, sh, opac, lc_v);
    make_cam(&cam, cam16, W, H, znear);
    make_wt(&wt, wkind, wpar);
    oproj* P = project_all(&S, &cam, &wt);
    if (!P) return 2;
    pix_ctx c = {P, n, &cam, &wt, xy, out_rgb, out_den, amb, amb_tau};
    run_parallel(render_pixels, &c, npix, nthreads);
    free(P);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Public: analytic gradient                                                 */
/*                                                                          */
/* Given G = dL/dC per pixel of rows [y_lo, y_hi), with C from Eq. 7 (the    */
/* loss depends on those rows only):                                        */
/*   dL/da_i(p)  = G_p . (c_i - C_p) / D_p                                  */
/*   dL/dc_i     = sum_p G_p a_i(p) / D_p                                   */
/*   dL/dc_B     = sum_p G_p w_B / D_p                                      */
/*   dL/dw_B     = sum_p G_p . (c_B - C_p) / D_p                            */
/* with D_p = w_B + sum_i a_i(p), a_i = u_i w_i g_i, g = exp(-q/2), and then */
/* the chain rule back through q, the conic, Sigma_2D, J, W, Sigma_3D, the   */
/* rotation, the scales, the SH and the weight functions.                   */
/*                                                                          */
/* Kinks (the derivative is taken as 0 on the flat side): max(0, .) in the   */
/* colour, max(0, .) in LC, the q <= 9 cutoff (a hard step, no derivative),  */
/* and the Jacobian clamp (the clamped coordinate does not move with t).    */
/*                                                                          */
/* Outputs (all overwritten): g_means[n*3], g_log_scales[n*3], g_quats[n*4], */
/* g_sh[n*K*3], g_opac[n or n*K], g_lc_v[n], g_wpar[6] (sigma, beta, w_B,    */
/* c_B), g2d[n*9]: per-Gaussian dL/d(mean2d x, y), dL/d(conic A, B, C),      */
/* dL/d(u w), dL/dc (3).  B is the off-diagonal conic entry, counted once.   */
/*                                                                          */
/* Tie bounds (optional, test infrastructure): an FP32 renderer may decide  */
/* pairs within rounding of the cutoff the other way (see tie_width), both  */
/* in its backward (which terms it sums) and in its forward (the C and D    */
/* the terms read).  To first order each gradient entry then moves by at    */
/* most                                                                     */
/*   B = sum over the Gaussian's tie pairs of |its term|                    */
/*     + sum over its other pairs at pixels holding ties of the term's      */
/*       change when C moves by amb and D by the tie mass m = sum |a|,      */
/* per g2d component, and each parameter entry by sum_k |chain_k| B_k, the  */
/* chain being linear in g2d; the background terms likewise per pixel.      */
/* ------------------------------------------------------------------------ */
typedef struct {
    const oscene* S; const oproj* P; const ocam* cam; const owt* wt;
    double cutoff;
    int y_lo, y_hi;          /* image rows covered by rgb, den and G */
    const double *rgb, *den, *G;
    double *g_means, *g_log_scales, *g_quats, *g_sh, *g_opac, *g_lc_v, *g2d;
    double gw[256][2];     /* per-thread partial sums: sigma, beta */
    /* tie bounds (NULL b_g2d: none) */
    const otie* tie;         /* per-pair windows from the FP32 model, or NULL for tie_tau */
    double tie_tau;
    const double *amb, *mass;   /* per pixel: the forward's tie allowance and tie mass */
    double *b_means, *b_log_scales, *b_quats, *b_sh, *b_opac, *b_lc_v, *b_g2d;
    double bw[256][2];
    int wide[256];
} grad_ctx;

/* One Gaussian's parameter gradients as the chain forms them from g2d. */
typedef struct {
    double means[3], log_scales[3], quats[4], sh[ORC_MAX_K * 3], opac[ORC_MAX_K], lc_v, sig, beta;
} ochain;

static void chain_one(const grad_ctx* c, long i, const double* g2, ochain* out)
{
    const oscene* S = c->S;
    const oproj* o = c->P + i;
    const ocam* cam = c->cam;
    const owt* wt = c->wt;
    const int K = S->K;
    memset(out, 0, sizeof *out);
    double gsig = 0, gbeta = 0;
    double g_t[3] = {0, 0, 0};      /* dL/dt (camera space) */
    double g_dir[3] = {0, 0, 0};    /* dL/d(unit direction) */
    double g_p[3] = {0, 0, 0};      /* dL/dp (world), direct terms */
    const double dL_duw = g2[5];
    const double dL_du = dL_duw * o->w, dL_dw = dL_duw * o->u;

    /* colour: c = max(0, Y.H + 0.5) */
    double Y[ORC_MAX_K], dY[ORC_MAX_K][3];
    sh_basis(S->deg, o->dir, Y, dY);
    const double* H = S->sh + (long)i * K * 3;
    double* gH = out->sh;
    for (int ch = 0; ch < 3; ++ch) {
        const double graw = (o->raw[ch] + 0.5 > 0) ? g2[6 + ch] : 0.0;
        for (int k = 0; k < K; ++k) {
            gH[3 * k + ch] = graw * Y[k];
            for (int e = 0; e < 3; ++e) g_dir[e] += graw * H[3 * k + ch] * dY[k][e];
        }
    }
    /* opacity */
    if (S->vd) {
        const double* Ha = S->opac + (long)i * K;
        double* gHa = out->opac;
        for (int k = 0; k < K; ++k) {
            gHa[k] = dL_du * Y[k];
            for (int e = 0; e < 3; ++e) g_dir[e] += dL_du * Ha[k] * dY[k][e];
        }
    } else {
        out->opac[0] = dL_du * o->u * (1.0 - o->u);
    }
    /* depth weight; d = t_z */
    const double d = o->d;
    double dL_dd = 0;
    if (wt->kind == 1) {
        const double db = pow(d, wt->beta);
        gsig += dL_dw * (-db) * o->w;
        gbeta += dL_dw * (-wt->sigma * db * log(d)) * o->w;
        dL_dd = dL_dw * (-wt->sigma * wt->beta * pow(d, wt->beta - 1.0)) * o->w;
    } else if (wt->kind == 2) {
        const double lin = 1.0 - d / wt->sigma;
        if (lin > 0) {
            const double v = S->lc_v[i];
            out->lc_v = dL_dw * lin;
            gsig += dL_dw * v * d / (wt->sigma * wt->sigma);
            dL_dd = dL_dw * (-v / wt->sigma);
        }
    }
    g_t[2] += dL_dd;
    /* direction: dir = v / |v| */
    {
        double dd = 0;
        for (int e = 0; e < 3; ++e) dd += o->dir[e] * g_dir[e];
        for (int e = 0; e < 3; ++e) g_p[e] += (g_dir[e] - o->dir[e] * dd) / o->vnorm;
    }
    /* projected mean */
    const double tx = o->t[0], ty = o->t[1], tz = o->t[2];
    g_t[0] += g2[0] * cam->fx / tz;
    g_t[1] += g2[1] * cam->fy / tz;
    g_t[2] += -g2[0] * cam->fx * tx / (tz * tz) - g2[1] * cam->fy * ty / (tz * tz);

    /* conic = Sigma_2D^{-1}:  dL/dSigma = -K Gk K with Gk the symmetric
     * matrix gradient [[gA, gB/2], [gB/2, gC]] */
    const double Kc[4] = {o->conic[0], o->conic[1], o->conic[1], o->conic[2]};
    const double Gk[4] = {g2[2], 0.5 * g2[3], 0.5 * g2[3], g2[4]};
    double t1[4], GS[4];
    mat_mul(Kc, Gk, t1, 2, 2, 2);
    mat_mul(t1, Kc, GS, 2, 2, 2);
    for (int e = 0; e < 4; ++e) GS[e] = -GS[e];
    /* Sigma_2D = T Sigma_3D T^t + 0.3 I,  T = J W */
    const double tanx = 0.5 * cam->W / cam->fx, tany = 0.5 * cam->H / cam->fy;
    const double limx = ORC_CLAMP * tanx, limy = ORC_CLAMP * tany;
    const double rx = clampd(tx / tz, -limx, limx), ry = clampd(ty / tz, -limy, limy);
    const int freex = (tx / tz >= -limx && tx / tz <= limx);
    const int freey = (ty / tz >= -limy && ty / tz <= limy);
    const double J[6] = {cam->fx / tz, 0, -cam->fx * rx / tz, 0, cam->fy / tz, -cam->fy * ry / tz};
    double T[6], Tt[6], Sig3[9], M[9], Mt[9], Rg[9];
    mat_mul(J, cam->R, T, 2, 3, 3);
    transpose(T, Tt, 2, 3);
    const double* qr = S->quats + 4 * i;
    const double qn = sqrt(qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3]);
    const double q[4] = {qr[0] / qn, qr[1] / qn, qr[2] / qn, qr[3] / qn};
    quat_to_rot(q, Rg);
    double s[3];
    for (int k = 0; k < 3; ++k) s[k] = exp(S->log_scales[3 * i + k]);
    for (int r = 0; r < 3; ++r)
        for (int cc = 0; cc < 3; ++cc) M[3 * r + cc] = Rg[3 * r + cc] * s[cc];
    transpose(M, Mt, 3, 3);
    mat_mul(M, Mt, Sig3, 3, 3, 3);
    /* dL/dSigma_3D = T^t GS T ;  dL/dT = 2 GS T Sigma_3D */
    double t2[6], GSig3[9], GT[6], t3[6];
    mat_mul(GS, T, t2, 2, 2, 3);
    mat_mul(Tt, t2, GSig3, 3, 2, 3);
    mat_mul(GS, T, t3, 2, 2, 3);
    mat_mul(t3, Sig3, GT, 2, 3, 3);
    for (int e = 0; e < 6; ++e) GT[e] *= 2.0;
    /* dL/dJ = dL/dT W^t */
    double Wt[9], GJ[6];
    transpose(cam->R, Wt, 3, 3);
    mat_mul(GT, Wt, GJ, 2, 3, 3);
    /* J00 = fx/tz, J02 = -fx rx/tz, J11 = fy/tz, J12 = -fy ry/tz,
     * rx = clamp(tx/tz) (moves with t only when not clamped) */
    g_t[2] += GJ[0] * (-cam->fx / (tz * tz)) + GJ[4] * (-cam->fy / (tz * tz));
    g_t[2] += GJ[2] * (cam->fx * rx / (tz * tz)) + GJ[5] * (cam->fy * ry / (tz * tz));
    if (freex) {
        g_t[0] += GJ[2] * (-cam->fx / (tz * tz));
        g_t[2] += GJ[2] * (-cam->fx / tz) * (-tx / (tz * tz));
    }
    if (freey) {
        g_t[1] += GJ[5] * (-cam->fy / (tz * tz));
        g_t[2] += GJ[5] * (-cam->fy / tz) * (-ty / (tz * tz));
    }
    /* t = W p + T  =>  dL/dp += W^t dL/dt */
    for (int e = 0; e < 3; ++e)
        g_p[e] += cam->R[e] * g_t[0] + cam->R[3 + e] * g_t[1] + cam->R[6 + e] * g_t[2];
    for (int e = 0; e < 3; ++e) out->means[e] = g_p[e];

    /* Sigma_3D = M M^t, M = R diag(s):  dL/dM = 2 dL/dSigma_3D M */
    double GM[9];
    mat_mul(GSig3, M, GM, 3, 3, 3);
    for (int e = 0; e < 9; ++e) GM[e] *= 2.0;
    double gs[3] = {0, 0, 0}, GR[9];
    for (int r = 0; r < 3; ++r)
        for (int cc = 0; cc < 3; ++cc) {
            GR[3 * r + cc] = GM[3 * r + cc] * s[cc];
            gs[cc] += GM[3 * r + cc] * Rg[3 * r + cc];
        }
    for (int k = 0; k < 3; ++k) out->log_scales[k] = gs[k] * s[k];
    /* rotation from the normalised quaternion */
    double dR[9][4], gqn[4] = {0, 0, 0, 0};
    quat_to_rot_grad(q, dR);
    for (int e = 0; e < 9; ++e)
        for (int k = 0; k < 4; ++k) gqn[k] += GR[e] * dR[e][k];
    double dot = 0;
    for (int k = 0; k < 4; ++k) dot += gqn[k] * q[k];
    for (int k = 0; k < 4; ++k) out->quats[k] = (gqn[k] - q[k] * dot) / qn;
    out->sig = gsig;
    out->beta = gbeta;
}

/* out (+)= s * |x| over n entries (s = 0: plain copy of x) */
static void put(double* out, const double* x, int n, double s)
{
    for (int k = 0; k < n; ++k) out[k] = s > 0 ? out[k] + s * fabs(x[k]) : x[k];
}

static void grad_gaussians(void* arg, long lo, long hi, int tid)
{
    grad_ctx* c = (grad_ctx*)arg;
    const oscene* S = c->S;
    const ocam* cam = c->cam;
    const int K = S->K, W = cam->W;
    const int nop = S->vd ? K : 1;
    const int bnd = c->b_g2d != NULL;
    double gsig = 0, gbeta = 0, bsig = 0, bbeta = 0;
    const double widest = c->tie ? ORC_TIE_CAP : c->tie_tau;
    for (long i = lo; i < hi; ++i) {
        const oproj* o = c->P + i;
        double* g2 = c->g2d + 9 * i;
        double B[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        memset(g2, 0, 9 * sizeof(double));
        if (!o->visible) {
            /* culled (behind the near plane): no gradient */
            ochain none;
            memset(&none, 0, sizeof none);
            put(c->g_means + 3 * i, none.means, 3, 0);
            put(c->g_log_scales + 3 * i, none.log_scales, 3, 0);
            put(c->g_quats + 4 * i, none.quats, 4, 0);
            put(c->g_sh + (long)i * K * 3, none.sh, K * 3, 0);
            put(c->g_opac + (long)i * nop, none.opac, nop, 0);
            c->g_lc_v[i] = 0;
            if (bnd) {
                put(c->b_means + 3 * i, none.means, 3, 0);
                put(c->b_log_scales + 3 * i, none.log_scales, 3, 0);
                put(c->b_quats + 4 * i, none.quats, 4, 0);
                put(c->b_sh + (long)i * K * 3, none.sh, K * 3, 0);
                put(c->b_opac + (long)i * nop, none.opac, nop, 0);
                c->b_lc_v[i] = 0;
                memset(c->b_g2d + 9 * i, 0, 9 * sizeof(double));
            }
            continue;
        }
        /* ---- per-pixel part: Eq. 7 and the Gaussian footprint ---- */
        int x0, x1, y0, y1;
        double reach = bnd && ORC_CUTOFF + widest > c->cutoff ? ORC_CUTOFF + widest : c->cutoff;
        if (orc_flip_seed[1] && ORC_CUTOFF + orc_flip_tau > reach) reach = ORC_CUTOFF + orc_flip_tau;
        pixel_range(o, cam, sqrt(reach / ORC_CUTOFF), &x0, &x1, &y0, &y1);
        if (y0 < c->y_lo) y0 = c->y_lo;
        if (y1 > c->y_hi - 1) y1 = c->y_hi - 1;
        const double uw = o->u * o->w;
        for (int y = y0; y <= y1; ++y)
            for (int x = x0; x <= x1; ++x) {
                const double dx = x + 0.5 - o->mean2d[0], dy = y + 0.5 - o->mean2d[1];
                const double q = quad_form(o->conic, dx, dy);
                const int in = counted(q, c->cutoff, i, x, y, 1);
                int tie = 0;
                if (bnd) {
                    const double tau = c->tie ? tie_width(c->tie + i, dx, dy, q, NULL) : c->tie_tau;
                    if (c->tie ? too_wide(q, tau) : tau > widest) c->wide[tid] = 1;
                    tie = fabs(q - ORC_CUTOFF) <= tau;
                }
                if (!in && !tie) continue;
                const long p = (long)(y - c->y_lo) * W + x;
                const double g = exp(-0.5 * q);
                const double a = uw * g;
                const double D = c->den[p];
                double dLda = 0, t[9];
                for (int ch = 0; ch < 3; ++ch) {
                    dLda += c->G[3 * p + ch] * (o->color[ch] - c->rgb[3 * p + ch]) / D;
                    t[6 + ch] = c->G[3 * p + ch] * a / D;                   /* dL/dc */
                }
                t[5] = dLda * g;                                           /* dL/d(uw) */
                const double dLdq = dLda * uw * (-0.5 * g);
                t[2] = dLdq * dx * dx;                                     /* dL/dA */
                t[3] = dLdq * 2.0 * dx * dy;                               /* dL/dB */
                t[4] = dLdq * dy * dy;                                     /* dL/dC */
                /* q depends on the mean through dx = px - mu */
                t[0] = dLdq * (-2.0) * (o->conic[0] * dx + o->conic[1] * dy);
                t[1] = dLdq * (-2.0) * (o->conic[1] * dx + o->conic[2] * dy);
                if (in)
                    for (int k = 0; k < 9; ++k) g2[k] += t[k];
                if (bnd && (tie || c->mass[p] > 0)) {
                    /* the forward's tie decisions move this pixel's C by at most amb and its D by at
                     * most the tie mass m, so |D'| >= dlo = |D| - m.  A tie pair's own term is at
                     * most its value at the worst such C and D; a counted pair's term moves by at
                     * most its change between (C, D) and the worst (C', D'). */
                    const double dlo = fabs(D) - c->mass[p];
                    double dla = 0, cw[3];
                    for (int ch = 0; ch < 3; ++ch) {
                        const double Gc = fabs(c->G[3 * p + ch]), e = fabs(o->color[ch] - c->rgb[3 * p + ch]);
                        if (tie) {
                            dla += Gc * (e + c->amb[p]) / dlo;
                            cw[ch] = Gc * fabs(a) / dlo;
                        } else {
                            dla += Gc * (c->amb[p] + e * c->mass[p] / fabs(D)) / dlo;
                            cw[ch] = Gc * fabs(a) * c->mass[p] / (fabs(D) * dlo);
                        }
                    }
                    if (!(dlo > 0)) dla = HUGE_VAL;
                    const double sq = fabs(uw) * 0.5 * g * dla;
                    B[5] += g * dla;
                    B[2] += sq * dx * dx;
                    B[3] += sq * 2.0 * fabs(dx * dy);
                    B[4] += sq * dy * dy;
                    B[0] += sq * 2.0 * fabs(o->conic[0] * dx + o->conic[1] * dy);
                    B[1] += sq * 2.0 * fabs(o->conic[1] * dx + o->conic[2] * dy);
                    for (int ch = 0; ch < 3; ++ch) B[6 + ch] += dlo > 0 ? cw[ch] : HUGE_VAL;
                }
            }

        /* ---- per-Gaussian chain ---- */
        ochain ch;
        chain_one(c, i, g2, &ch);
        put(c->g_means + 3 * i, ch.means, 3, 0);
        put(c->g_log_scales + 3 * i, ch.log_scales, 3, 0);
        put(c->g_quats + 4 * i, ch.quats, 4, 0);
        put(c->g_sh + (long)i * K * 3, ch.sh, K * 3, 0);
        put(c->g_opac + (long)i * nop, ch.opac, nop, 0);
        c->g_lc_v[i] = ch.lc_v;
        gsig += ch.sig;
        gbeta += ch.beta;
        if (!bnd) continue;
        memcpy(c->b_g2d + 9 * i, B, sizeof B);
        memset(c->b_means + 3 * i, 0, 3 * sizeof(double));
        memset(c->b_log_scales + 3 * i, 0, 3 * sizeof(double));
        memset(c->b_quats + 4 * i, 0, 4 * sizeof(double));
        memset(c->b_sh + (long)i * K * 3, 0, (size_t)K * 3 * sizeof(double));
        memset(c->b_opac + (long)i * nop, 0, (size_t)nop * sizeof(double));
        c->b_lc_v[i] = 0;
        for (int k = 0; k < 9; ++k) {
            if (!(B[k] > 0)) continue;
            double e[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            e[k] = 1.0;
            ochain ck;
            chain_one(c, i, e, &ck);
            put(c->b_means + 3 * i, ck.means, 3, B[k]);
            put(c->b_log_scales + 3 * i, ck.log_scales, 3, B[k]);
            put(c->b_quats + 4 * i, ck.quats, 4, B[k]);
            put(c->b_sh + (long)i * K * 3, ck.sh, K * 3, B[k]);
            put(c->b_opac + (long)i * nop, ck.opac, nop, B[k]);
            c->b_lc_v[i] += fabs(ck.lc_v) * B[k];
            bsig += fabs(ck.sig) * B[k];
            bbeta += fabs(ck.beta) * B[k];
        }
    }
    c->gw[tid][0] = gsig;
    c->gw[tid][1] = gbeta;
    c->bw[tid][0] = bsig;
    c->bw[tid][1] = bbeta;
}

/*
 * tie_tau: 0 for no tie bounds; > 0 for the window |q - 9| <= tie_tau for
 * every pair; < 0 for each pair's window from the FP32 rounding model.  With
 * tie bounds, b_* receive the bounds of the same shapes as g_* (b_wpar[6]).
 * Returns 3 if a model window broke the ORC_TIE_CAP rule (too_wide).
 */
int wsro_grad(long n, int deg, int vd, const double* means, const double* log_scales,
              const double* quats, const double* sh, const double* opac, const double* lc_v,
              const double* cam16, int W, int H, double znear, int wkind, const double* wpar,
              int nthreads, int y_lo, int y_hi, const double* grad_rgb,
              double* g_means, double* g_log_scales, double* g_quats, double* g_sh,
              double* g_opac, double* g_lc_v, double* g_wpar, double* g2d, double cutoff,
              double tie_tau, double* b_means, double* b_log_scales, double* b_quats, double* b_sh,
              double* b_opac, double* b_lc_v, double* b_wpar, double* b_g2d)
{
    if (deg < 0 || deg > 3 || n < 0 || W <= 0 || H <= 0) return 1;
    if (y_lo < 0 || y_hi > H || y_lo >= y_hi) return 1;
    const int bnd = tie_tau != 0.0;
    if (bnd && !(b_means && b_log_scales && b_quats && b_sh && b_opac && b_lc_v && b_wpar && b_g2d)) return 1;
    oscene S; ocam cam; owt wt;
    fill_scene(&S, n, deg, vd, means, log_scales, quats, sh, opac, lc_v);
    make_cam(&cam, cam16, W, H, znear);
    make_wt(&wt, wkind, wpar);
    const long np = (long)W * (y_hi - y_lo);
    double* rgb = (double*)malloc(np * 3 * sizeof(double));
    double* den = (double*)malloc(np * sizeof(double));
    double* amb = bnd ? (double*)malloc(np * sizeof(double)) : NULL;
    double* mass = bnd ? (double*)malloc(np * sizeof(double)) : NULL;
    if (!rgb || !den || (bnd && (!amb || !mass))) { free(rgb); free(den); free(amb); free(mass); return 2; }
    int rc = wsro_render(n, deg, vd, means, log_scales, quats, sh, opac, lc_v, cam16, W, H, znear,
                         wkind, wpar, nthreads, y_lo, y_hi, rgb, den, amb, tie_tau, NULL, cutoff, mass);
    if (rc) { free(rgb); free(den); free(amb); free(mass); return rc; }
    oproj* P = project_all(&S, &cam, &wt);
    grad_ctx* c = (grad_ctx*)calloc(1, sizeof(grad_ctx));
    otie* tm = (bnd && tie_tau < 0 && P) ? tie_all(&S, &cam, P) : NULL;
    if (!P || !c || (bnd && tie_tau < 0 && !tm)) {
        free(P); free(c); free(tm); free(rgb); free(den); free(amb); free(mass);
        return 2;
    }
    c->S = &S; c->P = P; c->cam = &cam; c->wt = &wt; c->y_lo = y_lo; c->y_hi = y_hi; c->cutoff = cutoff;
    c->rgb = rgb; c->den = den; c->G = grad_rgb;
    c->g_means = g_means; c->g_log_scales = g_log_scales; c->g_quats = g_quats; c->g_sh = g_sh;
    c->g_opac = g_opac; c->g_lc_v = g_lc_v; c->g2d = g2d;
    if (bnd) {
        c->tie = tm; c->tie_tau = tie_tau; c->amb = amb; c->mass = mass;
        c->b_means = b_means; c->b_log_scales = b_log_scales; c->b_quats = b_quats; c->b_sh = b_sh;
        c->b_opac = b_opac; c->b_lc_v = b_lc_v; c->b_g2d = b_g2d;
    }
    run_parallel(grad_gaussians, c, n, nthreads);
    for (int k = 0; k < 6; ++k) g_wpar[k] = 0;
    for (int t = 0; t < 256; ++t) { g_wpar[0] += c->gw[t][0]; g_wpar[1] += c->gw[t][1]; }
    if (bnd) {
        for (int k = 0; k < 6; ++k) b_wpar[k] = 0;
        for (int t = 0; t < 256; ++t) {
            b_wpar[0] += c->bw[t][0];
            b_wpar[1] += c->bw[t][1];
            if (c->wide[t]) rc = 3;
        }
    }
    /* background terms of Eq. 7 */
    for (long p = 0; p < np; ++p) {
        const double D = den[p];
        for (int ch = 0; ch < 3; ++ch) {
            g_wpar[2] += grad_rgb[3 * p + ch] * (wt.c_bg[ch] - rgb[3 * p + ch]) / D;
            g_wpar[3 + ch] += grad_rgb[3 * p + ch] * wt.w_bg / D;
            if (bnd && mass[p] > 0) {
                const double Gc = fabs(grad_rgb[3 * p + ch]), dlo = fabs(D) - mass[p];
                b_wpar[2] += dlo > 0 ? Gc * (amb[p] + fabs(wt.c_bg[ch] - rgb[3 * p + ch]) * mass[p] / fabs(D)) / dlo
                                     : HUGE_VAL;
                b_wpar[3 + ch] += dlo > 0 ? Gc * fabs(wt.w_bg) * mass[p] / (fabs(D) * dlo) : HUGE_VAL;
            }
        }
    }
    free(c); free(P); free(tm); free(rgb); free(den); free(amb); free(mass);
    return rc;
}

/*
 * The tie window of listed pairs (test infrastructure): for each k, the
 * Gaussian idx[k] at the pixel position (xy[2k], xy[2k+1]) (pixel units, not
 * a pixel index: any point).  Outputs: q[k] (exact), tau[k] (the window,
 * tie_width) and terms[6k .. 6k+5] (its parts: mean, rows, sums, record,
 * threshold, evaluation).
 */
int wsro_tie_width(long n, int deg, int vd, const double* means, const double* log_scales,
                   const double* quats, const double* sh, const double* opac, const double* lc_v,
                   const double* cam16, int W, int H, double znear, int wkind, const double* wpar,
                   long npts, const long* idx, const double* xy, double* q, double* tau, double* terms)
{
    if (deg < 0 || deg > 3 || n < 0) return 1;
    oscene S; ocam cam; owt wt;
    fill_scene(&S, n, deg, vd, means, log_scales, quats, sh, opac, lc_v);
    make_cam(&cam, cam16, W, H, znear);
    make_wt(&wt, wkind, wpar);
    for (long k = 0; k < npts; ++k) {
        if (idx[k] < 0 || idx[k] >= n) return 1;
        oproj o;
        otie m;
        project_one(&S, idx[k], &cam, &wt, &o);
        tie_model(&S, idx[k], &cam, &o, &m);
        if (!o.visible) {
            q[k] = tau[k] = -1.0;
            for (int j = 0; j < 6; ++j) terms[6 * k + j] = -1.0;
            continue;
        }
        const double dx = xy[2 * k] - o.mean2d[0], dy = xy[2 * k + 1] - o.mean2d[1];
        q[k] = quad_form(o.conic, dx, dy);
        tau[k] = tie_width(&m, dx, dy, q[k], terms + 6 * k);
    }
    return 0;
}
