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
} render_ctx;

static void render_rows(void* arg, long r0, long r1, int tid)
{
    render_ctx* c = (render_ctx*)arg;
    r0 += c->y_lo;
    r1 += c->y_lo;
    const int W = c->cam->W;
    long long pairs = 0;
    const double grow = sqrt((c->cutoff + (c->amb ? c->amb_tau : 0.0)) / ORC_CUTOFF);
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
                    if (fabs(q - c->cutoff) <= c->amb_tau) {
                        const double g = exp(-0.5 * q);
                        const double a = o->u * o->w * g;
                        double m = 0;
                        for (int ch = 0; ch < 3; ++ch) {
                            const double e = fabs(o->color[ch] - c->rgb[3 * p + ch]);
                            if (e > m) m = e;
                        }
                        c->amb[p] += fabs(a) * m / fabs(c->dent[p]);
                    }
                    continue;
                }
                if (q > c->cutoff) continue;
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
 * a bound on how far C can move if those pairs were decided the other way.
 * n_pairs (optional): number of (pixel, Gaussian) pairs with q <= 9.
 */
int wsro_render(long n, int deg, int vd, const double* means, const double* log_scales,
                const double* quats, const double* sh, const double* opac, const double* lc_v,
                const double* cam16, int W, int H, double znear, int wkind, const double* wpar,
                int nthreads, int y_lo, int y_hi, double* out_rgb, double* out_den, double* amb,
                double amb_tau, long long* n_pairs, double cutoff)
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
    render_ctx c = {P, n, &cam, &wt, cutoff, y_lo, num, den, pairs, amb_tau, NULL, NULL, NULL};
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
    if (amb) {
        memset(amb, 0, np * sizeof(double));
        render_ctx c2 = {P, n, &cam, &wt, cutoff, y_lo, NULL, NULL, pairs, amb_tau, amb, out_rgb, out_den};
        run_parallel(render_rows, &c2, rows, nthreads);
        for (long p = 0; p < np; ++p) amb[p] *= 1.05;
    }
    free(num); free(den); free(P);
    return 0;
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
        double am = 0;
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
                am += fabs(a) * m / fabs(D);
            }
            c->amb[k] = 1.05 * am;
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
/* ------------------------------------------------------------------------ */
typedef struct {
    const oscene* S; const oproj* P; const ocam* cam; const owt* wt;
    double cutoff;
    int y_lo, y_hi;          /* image rows covered by rgb, den and G */
    const double *rgb, *den, *G;
    double *g_means, *g_log_scales, *g_quats, *g_sh, *g_opac, *g_lc_v, *g2d;
    double gw[256][2];     /* per-thread partial sums: sigma, beta */
} grad_ctx;

static void grad_gaussians(void* arg, long lo, long hi, int tid)
{
    grad_ctx* c = (grad_ctx*)arg;
    const oscene* S = c->S;
    const ocam* cam = c->cam;
    const owt* wt = c->wt;
    const int K = S->K, W = cam->W;
    double gsig = 0, gbeta = 0;
    for (long i = lo; i < hi; ++i) {
        const oproj* o = c->P + i;
        double* g2 = c->g2d + 9 * i;
        memset(g2, 0, 9 * sizeof(double));
        if (!o->visible) continue;
        /* ---- per-pixel part: Eq. 7 and the Gaussian footprint ---- */
        int x0, x1, y0, y1;
        pixel_range(o, cam, sqrt(c->cutoff / ORC_CUTOFF), &x0, &x1, &y0, &y1);
        if (y0 < c->y_lo) y0 = c->y_lo;
        if (y1 > c->y_hi - 1) y1 = c->y_hi - 1;
        const double uw = o->u * o->w;
        for (int y = y0; y <= y1; ++y)
            for (int x = x0; x <= x1; ++x) {
                const double dx = x + 0.5 - o->mean2d[0], dy = y + 0.5 - o->mean2d[1];
                const double q = quad_form(o->conic, dx, dy);
                if (q > c->cutoff) continue;
                const long p = (long)(y - c->y_lo) * W + x;
                const double g = exp(-0.5 * q);
                const double a = uw * g;
                const double D = c->den[p];
                double dLda = 0;
                for (int ch = 0; ch < 3; ++ch) {
                    dLda += c->G[3 * p + ch] * (o->color[ch] - c->rgb[3 * p + ch]) / D;
                    g2[6 + ch] += c->G[3 * p + ch] * a / D;            /* dL/dc */
                }
                g2[5] += dLda * g;                                     /* dL/d(uw) */
                const double dLdq = dLda * uw * (-0.5 * g);
                g2[2] += dLdq * dx * dx;                               /* dL/dA */
                g2[3] += dLdq * 2.0 * dx * dy;                         /* dL/dB */
                g2[4] += dLdq * dy * dy;                               /* dL/dC */
                /* q depends on the mean through dx = px - mu */
                g2[0] += dLdq * (-2.0) * (o->conic[0] * dx + o->conic[1] * dy);
                g2[1] += dLdq * (-2.0) * (o->conic[1] * dx + o->conic[2] * dy);
            }

        /* ---- per-Gaussian chain ---- */
        double g_t[3] = {0, 0, 0};      /* dL/dt (camera space) */
        double g_dir[3] = {0, 0, 0};    /* dL/d(unit direction) */
        double g_p[3] = {0, 0, 0};      /* dL/dp (world), direct terms */
        const double dL_duw = g2[5];
        const double dL_du = dL_duw * o->w, dL_dw = dL_duw * o->u;

        /* colour: c = max(0, Y.H + 0.5) */
        double Y[ORC_MAX_K], dY[ORC_MAX_K][3];
        sh_basis(S->deg, o->dir, Y, dY);
        const double* H = S->sh + (long)i * K * 3;
        double* gH = c->g_sh + (long)i * K * 3;
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
            double* gHa = c->g_opac + (long)i * K;
            for (int k = 0; k < K; ++k) {
                gHa[k] = dL_du * Y[k];
                for (int e = 0; e < 3; ++e) g_dir[e] += dL_du * Ha[k] * dY[k][e];
            }
        } else {
            c->g_opac[i] = dL_du * o->u * (1.0 - o->u);
        }
        /* depth weight; d = t_z */
        const double d = o->d;
        double dL_dd = 0;
        c->g_lc_v[i] = 0;
        if (wt->kind == 1) {
            const double db = pow(d, wt->beta);
            gsig += dL_dw * (-db) * o->w;
            gbeta += dL_dw * (-wt->sigma * db * log(d)) * o->w;
            dL_dd = dL_dw * (-wt->sigma * wt->beta * pow(d, wt->beta - 1.0)) * o->w;
        } else if (wt->kind == 2) {
            const double lin = 1.0 - d / wt->sigma;
            if (lin > 0) {
                const double v = S->lc_v[i];
                c->g_lc_v[i] = dL_dw * lin;
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
        for (int e = 0; e < 3; ++e) c->g_means[3 * i + e] = g_p[e];

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
        for (int k = 0; k < 3; ++k) c->g_log_scales[3 * i + k] = gs[k] * s[k];
        /* rotation from the normalised quaternion */
        double dR[9][4], gqn[4] = {0, 0, 0, 0};
        quat_to_rot_grad(q, dR);
        for (int e = 0; e < 9; ++e)
            for (int k = 0; k < 4; ++k) gqn[k] += GR[e] * dR[e][k];
        double dot = 0;
        for (int k = 0; k < 4; ++k) dot += gqn[k] * q[k];
        for (int k = 0; k < 4; ++k) c->g_quats[4 * i + k] = (gqn[k] - q[k] * dot) / qn;
    }
    c->gw[tid][0] = gsig;
    c->gw[tid][1] = gbeta;
}

int wsro_grad(long n, int deg, int vd, const double* means, const double* log_scales,
              const double* quats, const double* sh, const double* opac, const double* lc_v,
              const double* cam16, int W, int H, double znear, int wkind, const double* wpar,
              int nthreads, int y_lo, int y_hi, const double* grad_rgb,
              double* g_means, double* g_log_scales, double* g_quats, double* g_sh,
              double* g_opac, double* g_lc_v, double* g_wpar, double* g2d, double cutoff)
{
    if (deg < 0 || deg > 3 || n < 0 || W <= 0 || H <= 0) return 1;
    if (y_lo < 0 || y_hi > H || y_lo >= y_hi) return 1;
    oscene S; ocam cam; owt wt;
    fill_scene(&S, n, deg, vd, means, log_scales, quats, sh, opac, lc_v);
    make_cam(&cam, cam16, W, H, znear);
    make_wt(&wt, wkind, wpar);
    const long np = (long)W * (y_hi - y_lo);
    double* rgb = (double*)malloc(np * 3 * sizeof(double));
    double* den = (double*)malloc(np * sizeof(double));
    if (!rgb || !den) { free(rgb); free(den); return 2; }
    int rc = wsro_render(n, deg, vd, means, log_scales, quats, sh, opac, lc_v, cam16, W, H, znear,
                         wkind, wpar, nthreads, y_lo, y_hi, rgb, den, NULL, 0.0, NULL, cutoff);
    if (rc) { free(rgb); free(den); return rc; }
    oproj* P = project_all(&S, &cam, &wt);
    if (!P) { free(rgb); free(den); return 2; }
    grad_ctx* c = (grad_ctx*)calloc(1, sizeof(grad_ctx));
    c->S = &S; c->P = P; c->cam = &cam; c->wt = &wt; c->y_lo = y_lo; c->y_hi = y_hi; c->cutoff = cutoff;
    c->rgb = rgb; c->den = den; c->G = grad_rgb;
    c->g_means = g_means; c->g_log_scales = g_log_scales; c->g_quats = g_quats; c->g_sh = g_sh;
    c->g_opac = g_opac; c->g_lc_v = g_lc_v; c->g2d = g2d;
    if (S.vd) memset(g_opac, 0, (size_t)n * S.K * sizeof(double));
    run_parallel(grad_gaussians, c, n, nthreads);
    for (int k = 0; k < 6; ++k) g_wpar[k] = 0;
    for (int t = 0; t < 256; ++t) { g_wpar[0] += c->gw[t][0]; g_wpar[1] += c->gw[t][1]; }
    /* background terms of Eq. 7 */
    for (long p = 0; p < np; ++p) {
        const double D = den[p];
        for (int ch = 0; ch < 3; ++ch) {
            g_wpar[2] += grad_rgb[3 * p + ch] * (wt.c_bg[ch] - rgb[3 * p + ch]) / D;
            g_wpar[3 + ch] += grad_rgb[3 * p + ch] * wt.w_bg / D;
        }
    }
    /* invisible Gaussians: zero gradients */
    for (long i = 0; i < n; ++i)
        if (!P[i].visible) {
            memset(g_means + 3 * i, 0, 3 * sizeof(double));
            memset(g_log_scales + 3 * i, 0, 3 * sizeof(double));
            memset(g_quats + 4 * i, 0, 4 * sizeof(double));
            memset(g_sh + (long)i * S.K * 3, 0, (size_t)S.K * 3 * sizeof(double));
            if (S.vd) memset(g_opac + (long)i * S.K, 0, (size_t)S.K * sizeof(double));
            else g_opac[i] = 0;
            g_lc_v[i] = 0;
        }
    free(c); free(P); free(rgb); free(den);
    return 0;
}
