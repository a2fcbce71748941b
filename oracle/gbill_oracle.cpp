/*
 * gbill_oracle.cpp -- plain, slow FP64 CPU oracle for the textured 2D-Gaussian
 * surfel rasterizer of "Gaussian Billboards: Expressive 2D Gaussian Splatting
 * with Textures" (arXiv 2412.12734).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code:
 * only the test-suite, the smoke check and the CPU-baseline leg of the bench
 * load it.  It shares no source, header, constant table or helper with the
 * CUDA library; the only thing both sides see is the seeded input arrays.
 *
 * What it computes, in the paper's order:
 *   - 2DGS primitive: centre p, tangents t_u, t_v taken from a unit quaternion,
 *     scales (s_u, s_v)                                  (Sec. 3.1, Eq. 3)
 *   - uv-space Gaussian G(u,v) = exp(-(u^2+v^2)/2)       (Sec. 3.1, Eq. 4)
 *   - colour grid C_k (N x N x 3) over [-sigma, sigma]^2, sampled with the
 *     border-clamped bilinear lookup                     (Sec. 3.2, Eq. 5, Alg. 2)
 *   - one per-splat set of SH coefficients added on top of the grid colour
 *     (diffuse/specular split)                           (Sec. 4.2)
 *   - front-to-back alpha compositing                    (Sec. 3.1, Eq. 2, Alg. 1)
 *   - backward: reverse walk from the final transmittance with the colour
 *     adjoint through adj-bilinear                       (Alg. 1 bwd, Alg. 2)
 *
 * Readings of points the paper leaves open (each one is listed in the design
 * notes of the repository, same numbering):
 *   R1/R2  bilinear index: i = min(floor(u'), N-2), f = u' - i; N = 1 is the
 *          constant colour C[0,0] with zero uv adjoint.
 *   R3     adj-bilinear accumulates (+=) into the grid gradient.
 *   R4     uv adjoint mask is the strict -sigma < u < sigma.
 *   R5/R6  grid layout [K][i_u][i_v][3], corner aligned over [-sigma, sigma].
 *   R7     colour = bilinear(C) + sum_lm k_lm Y_lm(d), no offset, no clamp.
 *   R8     real SH up to degree 3 with the (-1)^m sign convention.
 *   R9     ray/splat intersection: zeta = adj(T) (x, y, 1), u = zeta_x/zeta_z.
 *   R10    screen-space low-pass: rho = min(u^2+v^2, 2 |x - c|^2); a tie goes
 *          to the uv branch; depth is the plane-hit depth on the uv branch and
 *          the centre depth on the low-pass branch.
 *   R11    alpha = min(0.99, o G); skip alpha < 1/255; stop before a splat when
 *          T (1 - alpha) < 1e-4.
 *   R12    pixel (x, y) has its centre at (x + 0.5, y + 0.5).
 *   R14-16 culling, tile rectangles and the depth key are FP32 decisions; both
 *          sides take them in FP32 (key_formula_f32 below), and the oracle's
 *          explicit depth sort orders splats by (FP32 depth bits, splat id).
 *   R17    optional background added as T_final * bg.
 *   R18    depth output = sum_i z_i alpha_i T_i (not normalised).
 *   R28    per-splat grid size n_k <= N: splat k's grid is rows and columns
 *          0..n_k-1 of its N x N block, sampled by Alg. 2 with n_k.
 *
 * Build: g++ -O2 -std=c++17 -ffp-contract=off -fPIC -shared -pthread
 * (-ffp-contract=off keeps the FP32 key formula free of fused multiply-adds.)
 */
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

extern "C" {

/* ------------------------------------------------------------------------ */
/* Public structures (mirrored by the ctypes wrapper in oracle/__init__.py)  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t num_splats;
    const double *means;      /* [K,3]                                      */
    const double *quats;      /* [K,4] (w, x, y, z), any positive norm       */
    const double *scales;     /* [K,2] linear (s_u, s_v)                     */
    const double *opacities;  /* [K]   in (0, 1)                             */
    const double *sh;         /* [K,(D+1)^2,3]                               */
    const double *textures;   /* [K,N,N,3]  C[i_u][i_v][c]                   */
    int32_t sh_degree;        /* D in 0..3                                   */
    int32_t tex_n;            /* N >= 1                                      */
    double sigma;             /* grid extent, default 0.5                    */
    const int32_t *splat_n;   /* [K] or NULL: splat k's grid is n_k x n_k,    */
                              /* 1 <= n_k <= N, in rows and columns 0..n_k-1 */
                              /* of its N x N block (Alg. 2 with n_k)         */
} orc_scene;

typedef struct {
    int32_t width, height;
    double fx, fy, cx, cy;
    double w2c[12];           /* row-major 3x4 [R | t], OpenCV axes          */
    double near_plane;
} orc_camera;

/* Pixel window [x0, x0+w) x [y0, y0+h) of one view. */
typedef struct { int32_t x0, y0, w, h; } orc_window;

/* Per-pixel forward outputs inside the window (row-major w*h). */
typedef struct {
    double *rgb;          /* [h*w*3] */
    double *depth;        /* [h*w]   */
    double *alpha;        /* [h*w]   */
    double *t_final;      /* [h*w]   */
    int32_t *n_contrib;   /* [h*w] number of splats blended                  */
    double *margin_fwd;   /* [h*w] min relative distance of a forward-        */
                          /*       discontinuous decision to its threshold  */
    double *margin_grad;  /* [h*w] same over every decision with a kink      */
    int64_t *n_pairs;     /* [1]   pairs evaluated                           */
} orc_fwd_out;

typedef struct {
    double *d_means;      /* [K,3]           accumulated (+=) */
    double *d_quats;      /* [K,4]           */
    double *d_scales;     /* [K,2]           */
    double *d_opacities;  /* [K]             */
    double *d_sh;         /* [K,(D+1)^2,3]   */
    double *d_textures;   /* [K,N,N,3]       */
} orc_grads;

/* ------------------------------------------------------------------------ */
/* Constants of the method                                                  */
/* ------------------------------------------------------------------------ */

static const double kAlphaMin = 1.0 / 255.0;   /* R11 */
static const double kAlphaMax = 0.99;          /* R11 */
static const double kTMin = 1e-4;              /* R11 */
static const double kLowPass = 2.0;            /* R10: 1 / (sqrt(2)/2)^2 */

/* FP32 literals of the tile formula (R15).  rho_max = 2 ln 255 bounds
 * u^2+v^2 wherever alpha >= 1/255 can hold (o <= 1);  the low-pass disk
 * radius is sqrt(rho_max / 2) = sqrt(ln 255). */
static const float kRhoMaxF = 11.0825270903f;
static const float kLowPassRadiusF = 2.35398885833f;

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics, degree <= 3  (R8)                              */
/* Y_lm for m = -l..l, written as polynomials in the unit direction d; the  */
/* sign is (-1)^m times the usual real basis.  Constants follow from        */
/* N_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) and the associated Legendre */
/* polynomials; they are evaluated here from that definition.               */
/* ------------------------------------------------------------------------ */

static void sh_eval(int D, const double d[3], double *Y, double (*dY)[3]) {
    const double pi = 3.14159265358979323846;
    const double x = d[0], y = d[1], z = d[2];
    const double c0 = 0.5 * std::sqrt(1.0 / pi);
    const double c1 = std::sqrt(3.0 / (4.0 * pi));
    const double c2a = 0.5 * std::sqrt(15.0 / pi);
    const double c2b = 0.25 * std::sqrt(5.0 / pi);
    const double c2c = 0.25 * std::sqrt(15.0 / pi);
    const double c3a = 0.25 * std::sqrt(35.0 / (2.0 * pi));
    const double c3b = 0.5 * std::sqrt(105.0 / pi);
    const double c3c = 0.25 * std::sqrt(21.0 / (2.0 * pi));
    const double c3d = 0.25 * std::sqrt(7.0 / pi);
    const double c3e = 0.25 * std::sqrt(105.0 / pi);
    int i = 0;
    auto put = [&](double v, double gx, double gy, double gz) {
        Y[i] = v;
        if (dY) { dY[i][0] = gx; dY[i][1] = gy; dY[i][2] = gz; }
        ++i;
    };
    put(c0, 0, 0, 0);
    if (D >= 1) {
        put(-c1 * y, 0, -c1, 0);
        put(c1 * z, 0, 0, c1);
        put(-c1 * x, -c1, 0, 0);
    }
    if (D >= 2) {
        put(c2a * x * y, c2a * y, c2a * x, 0);
        put(-c2a * y * z, 0, -c2a * z, -c2a * y);
        put(c2b * (2 * z * z - x * x - y * y), -2 * c2b * x, -2 * c2b * y, 4 * c2b * z);
        put(-c2a * x * z, -c2a * z, 0, -c2a * x);
        put(c2c * (x * x - y * y), 2 * c2c * x, -2 * c2c * y, 0);
    }
    if (D >= 3) {
        put(-c3a * y * (3 * x * x - y * y), -c3a * 6 * x * y, -c3a * (3 * x * x - 3 * y * y), 0);
        put(c3b * x * y * z, c3b * y * z, c3b * x * z, c3b * x * y);
        put(-c3c * y * (4 * z * z - x * x - y * y), -c3c * (-2 * x * y),
            -c3c * (4 * z * z - x * x - 3 * y * y), -c3c * 8 * y * z);
        put(c3d * z * (2 * z * z - 3 * x * x - 3 * y * y), c3d * (-6 * x * z), c3d * (-6 * y * z),
            c3d * (6 * z * z - 3 * x * x - 3 * y * y));
        put(-c3c * x * (4 * z * z - x * x - y * y), -c3c * (4 * z * z - 3 * x * x - y * y),
            -c3c * (-2 * x * y), -c3c * 8 * x * z);
        put(c3e * z * (x * x - y * y), c3e * 2 * x * z, -c3e * 2 * y * z, c3e * (x * x - y * y));
        put(-c3a * x * (x * x - 3 * y * y), -c3a * (3 * x * x - 3 * y * y), -c3a * (-6 * x * y), 0);
    }
}

/* ------------------------------------------------------------------------ */
/* Alg. 2: bilinear and adj-bilinear  (R1-R6)                               */
/* ------------------------------------------------------------------------ */

struct Bilin {
    int iu, iv;
    double fu, fv;
};

static Bilin bilin_coords(double u, double v, int N, double sigma) {
    Bilin b;
    double up = (N - 1) * (u + sigma) / (2.0 * sigma);
    double vp = (N - 1) * (v + sigma) / (2.0 * sigma);
    up = std::min(std::max(up, 0.0), double(N - 1));
    vp = std::min(std::max(vp, 0.0), double(N - 1));
    if (N == 1) { b.iu = b.iv = 0; b.fu = b.fv = 0.0; return b; }
    b.iu = std::min(int(std::floor(up)), N - 2);
    b.iv = std::min(int(std::floor(vp)), N - 2);
    b.fu = up - b.iu;
    b.fv = vp - b.iv;
    return b;
}

/* C: the grid's texel (i_u, i_v) at C + (i_u * stride + i_v) * 3; stride = N
   unless the grid is the leading N x N part of a larger block. */
static void bilinear(double u, double v, int N, double sigma, const double *C, double out[3], int stride = 0) {
    if (stride == 0) stride = N;
    Bilin b = bilin_coords(u, v, N, sigma);
    if (N == 1) { for (int c = 0; c < 3; ++c) out[c] = C[c]; return; }
    const double *c00 = C + ((b.iu) * stride + b.iv) * 3;
    const double *c10 = C + ((b.iu + 1) * stride + b.iv) * 3;
    const double *c01 = C + ((b.iu) * stride + b.iv + 1) * 3;
    const double *c11 = C + ((b.iu + 1) * stride + b.iv + 1) * 3;
    for (int c = 0; c < 3; ++c)
        out[c] = c00[c] * (1 - b.fu) * (1 - b.fv) + c10[c] * b.fu * (1 - b.fv) +
                 c01[c] * (1 - b.fu) * b.fv + c11[c] * b.fu * b.fv;
}

/* Adds the grid adjoint into Chat; returns the uv adjoint in uv_hat. */
static void adj_bilinear(double u, double v, int N, double sigma, const double *C,
                         const double chat[3], double *Chat, double uv_hat[2], int stride = 0) {
    if (stride == 0) stride = N;
    Bilin b = bilin_coords(u, v, N, sigma);
    if (N == 1) {
        for (int c = 0; c < 3; ++c) Chat[c] += chat[c];
        uv_hat[0] = uv_hat[1] = 0.0;
        return;
    }
    const int i00 = ((b.iu) * stride + b.iv) * 3, i10 = ((b.iu + 1) * stride + b.iv) * 3;
    const int i01 = ((b.iu) * stride + b.iv + 1) * 3, i11 = ((b.iu + 1) * stride + b.iv + 1) * 3;
    double fu_hat = 0.0, fv_hat = 0.0;
    for (int c = 0; c < 3; ++c) {
        Chat[i00 + c] += chat[c] * (1 - b.fu) * (1 - b.fv);
        Chat[i10 + c] += chat[c] * b.fu * (1 - b.fv);
        Chat[i01 + c] += chat[c] * (1 - b.fu) * b.fv;
        Chat[i11 + c] += chat[c] * b.fu * b.fv;
        fu_hat += chat[c] * ((C[i10 + c] - C[i00 + c]) * (1 - b.fv) + (C[i11 + c] - C[i01 + c]) * b.fv);
        fv_hat += chat[c] * ((C[i01 + c] - C[i00 + c]) * (1 - b.fu) + (C[i11 + c] - C[i10 + c]) * b.fu);
    }
    const double k = (N - 1) / (2.0 * sigma);
    uv_hat[0] = (u > -sigma && u < sigma) ? k * fu_hat : 0.0;
    uv_hat[1] = (v > -sigma && v < sigma) ? k * fv_hat : 0.0;
}

/* ------------------------------------------------------------------------ */
/* FP32 tile-rectangle and depth-key formula (R14-R16).                     */
/* Every operation is a single IEEE FP32 operation in the order written;    */
/* the library computes the same sequence, so culling, rectangles and keys  */
/* agree bit for bit.                                                        */
/* ------------------------------------------------------------------------ */

static int key_formula_f32(const float p[3], const float q[4], const float s[2], float o,
                           const float Rc[9], const float tc[3], float fx, float fy, float cxk,
                           float cyk, int W, int H, float near_plane, float *z_out,
                           int prect[4]) {
    const float qn2 = ((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3];
    if (!(qn2 > 0.0f)) return 0;
    const float qinv = 1.0f / std::sqrt(qn2);
    const float w = q[0] * qinv, x = q[1] * qinv, y = q[2] * qinv, z = q[3] * qinv;
    /* first two columns of the rotation matrix of (w, x, y, z) */
    const float tu0 = 1.0f - 2.0f * (y * y + z * z);
    const float tu1 = 2.0f * (x * y + w * z);
    const float tu2 = 2.0f * (x * z - w * y);
    const float tv0 = 2.0f * (x * y - w * z);
    const float tv1 = 1.0f - 2.0f * (x * x + z * z);
    const float tv2 = 2.0f * (y * z + w * x);
    const float a0 = s[0] * tu0, a1 = s[0] * tu1, a2 = s[0] * tu2;
    const float b0 = s[1] * tv0, b1 = s[1] * tv1, b2 = s[1] * tv2;
    const float A0 = (Rc[0] * a0 + Rc[1] * a1) + Rc[2] * a2;
    const float A1 = (Rc[3] * a0 + Rc[4] * a1) + Rc[5] * a2;
    const float A2 = (Rc[6] * a0 + Rc[7] * a1) + Rc[8] * a2;
    const float B0 = (Rc[0] * b0 + Rc[1] * b1) + Rc[2] * b2;
    const float B1 = (Rc[3] * b0 + Rc[4] * b1) + Rc[5] * b2;
    const float B2 = (Rc[6] * b0 + Rc[7] * b1) + Rc[8] * b2;
    const float P0 = ((Rc[0] * p[0] + Rc[1] * p[1]) + Rc[2] * p[2]) + tc[0];
    const float P1 = ((Rc[3] * p[0] + Rc[4] * p[1]) + Rc[5] * p[2]) + tc[1];
    const float P2 = ((Rc[6] * p[0] + Rc[7] * p[1]) + Rc[8] * p[2]) + tc[2];
    if (!(P2 > near_plane)) return 0;
    if (!(o >= 1.0f / 255.0f)) return 0;
    /* homography with the projected centre moved to the origin */
    const float xz = P0 / P2, yz = P1 / P2;
    const float t00 = fx * (A0 - A2 * xz), t01 = fx * (B0 - B2 * xz);
    const float t10 = fy * (A1 - A2 * yz), t11 = fy * (B1 - B2 * yz);
    const float t20 = A2, t21 = B2;
    /* dual conic of u^2+v^2 = rho_max:  T' diag(rho, rho, -1) T'^T */
    const float d00 = kRhoMaxF * (t00 * t00 + t01 * t01);
    const float d11 = kRhoMaxF * (t10 * t10 + t11 * t11);
    const float d02 = kRhoMaxF * (t00 * t20 + t01 * t21);
    const float d12 = kRhoMaxF * (t10 * t20 + t11 * t21);
    const float d22 = kRhoMaxF * (t20 * t20 + t21 * t21) - P2 * P2;
    if (!(d22 < 0.0f)) return 0; /* ellipse not bounded in front of the camera */
    const float nd = -d22;
    const float ox = d02 / d22, oy = d12 / d22;
    const float hx = std::sqrt(d02 * d02 + d00 * nd) / nd;
    const float hy = std::sqrt(d12 * d12 + d11 * nd) / nd;
    const float cx = fx * xz + cxk, cy = fy * yz + cyk;
    float elx = (cx + ox) - hx, ehx = (cx + ox) + hx;
    float ely = (cy + oy) - hy, ehy = (cy + oy) + hy;
    if (!(elx == elx) || !(ehx == ehx)) { elx = -INFINITY; ehx = INFINITY; }
    if (!(ely == ely) || !(ehy == ehy)) { ely = -INFINITY; ehy = INFINITY; }
    const float lox = std::fmin(elx, cx - kLowPassRadiusF), hix = std::fmax(ehx, cx + kLowPassRadiusF);
    const float loy = std::fmin(ely, cy - kLowPassRadiusF), hiy = std::fmax(ehy, cy + kLowPassRadiusF);
    /* pixel x covers centre x + 0.5:  x in [ceil(lo - 0.5), floor(hi - 0.5)] */
    const float fx0 = std::fmax(std::ceil(lox - 0.5f), 0.0f);
    const float fx1 = std::fmin(std::floor(hix - 0.5f), float(W - 1));
    const float fy0 = std::fmax(std::ceil(loy - 0.5f), 0.0f);
    const float fy1 = std::fmin(std::floor(hiy - 0.5f), float(H - 1));
    if (!(fx0 <= fx1) || !(fy0 <= fy1)) return 0;
    prect[0] = int(fx0);
    prect[1] = int(fy0);
    prect[2] = int(fx1);
    prect[3] = int(fy1);
    *z_out = P2;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* FP64 per-splat projection                                                */
/* ------------------------------------------------------------------------ */

struct Proj {
    double T[9];      /* T = K [R|t] [s_u t_u, s_v t_v, p], row-major */
    double adj[9];    /* adj(T) */
    double c[2];      /* projected centre (T02/T22, T12/T22)           */
    double rgb_sh[3]; /* SH colour                                      */
    double dir[3];    /* unit view direction (p - cam)/|p - cam|        */
    double dist;      /* |p - cam|                                      */
    double tu[3], tv[3], Rm[9]; /* tangent frame                        */
    double qn[4], qnorm;
};

static void quat_to_rot(const double qn[4], double R[9]) {
    const double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

static void adjugate3(const double T[9], double A[9]) {
    /* adj(T)[i][j] = cofactor of T[j][i] */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const int r1 = (j + 1) % 3, r2 = (j + 2) % 3, c1 = (i + 1) % 3, c2 = (i + 2) % 3;
            A[i * 3 + j] = T[r1 * 3 + c1] * T[r2 * 3 + c2] - T[r1 * 3 + c2] * T[r2 * 3 + c1];
        }
}

static void project(const orc_scene &sc, const orc_camera &cam, int64_t k, Proj &pr) {
    const double *p = sc.means + 3 * k, *q = sc.quats + 4 * k, *s = sc.scales + 2 * k;
    pr.qnorm = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; ++i) pr.qn[i] = q[i] / pr.qnorm;
    quat_to_rot(pr.qn, pr.Rm);
    for (int i = 0; i < 3; ++i) { pr.tu[i] = pr.Rm[i * 3 + 0]; pr.tv[i] = pr.Rm[i * 3 + 1]; }
    /* columns of the splat-to-world map (Eq. 3): s_u t_u, s_v t_v, p */
    double H[3][3];
    for (int i = 0; i < 3; ++i) { H[0][i] = s[0] * pr.tu[i]; H[1][i] = s[1] * pr.tv[i]; H[2][i] = p[i]; }
    const double *W = cam.w2c;
    double camcol[3][3]; /* camera-space columns: R a, R b, R p + t */
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) {
            camcol[j][i] = W[i * 4 + 0] * H[j][0] + W[i * 4 + 1] * H[j][1] + W[i * 4 + 2] * H[j][2];
            if (j == 2) camcol[j][i] += W[i * 4 + 3];
        }
    for (int j = 0; j < 3; ++j) {
        pr.T[0 * 3 + j] = cam.fx * camcol[j][0] + cam.cx * camcol[j][2];
        pr.T[1 * 3 + j] = cam.fy * camcol[j][1] + cam.cy * camcol[j][2];
        pr.T[2 * 3 + j] = camcol[j][2];
    }
    adjugate3(pr.T, pr.adj);
    pr.c[0] = pr.T[2] / pr.T[8];
    pr.c[1] = pr.T[5] / pr.T[8];
    /* camera position -R^T t and view direction */
    double campos[3];
    for (int i = 0; i < 3; ++i)
        campos[i] = -(W[0 * 4 + i] * W[3] + W[1 * 4 + i] * W[7] + W[2 * 4 + i] * W[11]);
    double d[3] = {p[0] - campos[0], p[1] - campos[1], p[2] - campos[2]};
    pr.dist = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int i = 0; i < 3; ++i) pr.dir[i] = d[i] / pr.dist;
    const int M = (sc.sh_degree + 1) * (sc.sh_degree + 1);
    double Y[16];
    sh_eval(sc.sh_degree, pr.dir, Y, nullptr);
    const double *kk = sc.sh + k * M * 3;
    for (int c = 0; c < 3; ++c) {
        double acc = 0.0;
        for (int m = 0; m < M; ++m) acc += kk[m * 3 + c] * Y[m];
        pr.rgb_sh[c] = acc;
    }
}

/* FP32 decision for splat k in camera cam (R14-R16). */
static int splat_key(const orc_scene &sc, const orc_camera &cam, int64_t k, float *z, int prect[4]) {
    float p[3], q[4], s[2], Rc[9], tc[3];
    for (int i = 0; i < 3; ++i) p[i] = float(sc.means[3 * k + i]);
    for (int i = 0; i < 4; ++i) q[i] = float(sc.quats[4 * k + i]);
    for (int i = 0; i < 2; ++i) s[i] = float(sc.scales[2 * k + i]);
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) Rc[i * 3 + j] = float(cam.w2c[i * 4 + j]);
        tc[i] = float(cam.w2c[i * 4 + 3]);
    }
    return key_formula_f32(p, q, s, float(sc.opacities[k]), Rc, tc, float(cam.fx), float(cam.fy),
                           float(cam.cx), float(cam.cy), cam.width, cam.height,
                           float(cam.near_plane), z, prect);
}

static uint32_t float_bits(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u;
}

/* Explicit depth sort: the non-culled splats ordered by (FP32 depth bits, id). */
static std::vector<int64_t> depth_order(const orc_scene &sc, const orc_camera &cam,
                                        std::vector<std::array<int, 4>> *rects) {
    std::vector<std::pair<uint32_t, int64_t>> v;
    if (rects) rects->assign(sc.num_splats, {0, 0, -1, -1});
    for (int64_t k = 0; k < sc.num_splats; ++k) {
        float z;
        int r[4];
        if (splat_key(sc, cam, k, &z, r)) {
            v.push_back({float_bits(z), k});
            if (rects) (*rects)[k] = {r[0], r[1], r[2], r[3]};
        }
    }
    std::stable_sort(v.begin(), v.end(),
                     [](const std::pair<uint32_t, int64_t> &a, const std::pair<uint32_t, int64_t> &b) {
                         return a.first < b.first;
                     });
    std::vector<int64_t> order;
    order.reserve(v.size());
    for (auto &e : v) order.push_back(e.second);
    return order;
}

/* ------------------------------------------------------------------------ */
/* Per-pixel evaluation of one splat (Eq. 4, Eq. 5, R9-R11)                 */
/* ------------------------------------------------------------------------ */

struct PairEval {
    bool hit;        /* zeta_z != 0 */
    double zeta[3], u, v, rho_uv, rho_lp, rho, G, alpha_raw, alpha, dx, dy;
    bool uv_branch, clamped;
};

static void eval_pair(const Proj &pr, double opac, double px, double py, PairEval &e) {
    const double *A = pr.adj;
    e.zeta[0] = A[0] * px + A[1] * py + A[2];
    e.zeta[1] = A[3] * px + A[4] * py + A[5];
    e.zeta[2] = A[6] * px + A[7] * py + A[8];
    e.hit = e.zeta[2] != 0.0;
    if (!e.hit) return;
    e.u = e.zeta[0] / e.zeta[2];
    e.v = e.zeta[1] / e.zeta[2];
    e.rho_uv = e.u * e.u + e.v * e.v;
    e.dx = px - pr.c[0];
    e.dy = py - pr.c[1];
    e.rho_lp = kLowPass * (e.dx * e.dx + e.dy * e.dy);
    e.uv_branch = e.rho_uv <= e.rho_lp;
    e.rho = e.uv_branch ? e.rho_uv : e.rho_lp;
    e.G = std::exp(-0.5 * e.rho);
    e.alpha_raw = opac * e.G;
    e.clamped = e.alpha_raw > kAlphaMax;
    e.alpha = e.clamped ? kAlphaMax : e.alpha_raw;
}

static double reldist(double a, double thr) { return std::fabs(a - thr) / std::fabs(thr); }

/* ------------------------------------------------------------------------ */
/* Conservative FP64 bounding box used only to skip far pairs (prefilter).  */
/* ------------------------------------------------------------------------ */

static void bbox64(const Proj &pr, double rho, double out[4]) {
    const double *T = pr.T;
    /* dual conic T diag(rho, rho, -1) T^T */
    auto Dij = [&](int i, int j) {
        return rho * (T[i * 3 + 0] * T[j * 3 + 0] + T[i * 3 + 1] * T[j * 3 + 1]) - T[i * 3 + 2] * T[j * 3 + 2];
    };
    const double d00 = Dij(0, 0), d11 = Dij(1, 1), d02 = Dij(0, 2), d12 = Dij(1, 2), d22 = Dij(2, 2);
    const double r = std::sqrt(rho / kLowPass);
    double lx = pr.c[0] - r, hx = pr.c[0] + r, ly = pr.c[1] - r, hy = pr.c[1] + r;
    if (d22 < 0) {
        const double ex = d02 / d22, ey = d12 / d22;
        const double wx = std::sqrt(std::max(0.0, d02 * d02 - d00 * d22)) / -d22;
        const double wy = std::sqrt(std::max(0.0, d12 * d12 - d11 * d22)) / -d22;
        lx = std::min(lx, ex - wx); hx = std::max(hx, ex + wx);
        ly = std::min(ly, ey - wy); hy = std::max(hy, ey + wy);
    } else {
        lx = ly = -INFINITY; hx = hy = INFINITY;
    }
    out[0] = lx; out[1] = ly; out[2] = hx; out[3] = hy;
}

/* ------------------------------------------------------------------------ */
/* Forward (Alg. 1 fwd, brute force over every splat at every pixel)        */
/* ------------------------------------------------------------------------ */

struct Contrib {
    int64_t k;
    PairEval e;
    double T;        /* transmittance before this splat */
    double col[3];   /* grid colour + SH colour         */
    double zi;       /* depth of this contribution      */
};

struct Ctx {
    const orc_scene *sc;
    const orc_camera *cam;
    std::vector<int64_t> order;
    std::vector<Proj> proj;          /* indexed by position in order */
    std::vector<std::array<double, 4>> box; /* prefilter boxes       */
    bool prefilter;
    double bg[3];
    /* prefilter bins: 16x16-pixel cells listing (in depth order) the splats
       whose box touches the cell; the per-pixel box test stays exact */
    int bins_x = 0, bins_y = 0;
    std::vector<std::vector<int32_t>> bins;
};

/* Runs the front-to-back loop of one pixel; fills the contributor list. */
static void pixel_forward(const Ctx &cx, int px, int py, std::vector<Contrib> *contribs,
                          double rgb[3], double *depth, double *t_final, int *n_contrib,
                          double *mfwd, double *mgrad, int64_t *npairs) {
    const orc_scene &sc = *cx.sc;
    const double X = px + 0.5, Y = py + 0.5;
    const int N = sc.tex_n;
    double T = 1.0, C[3] = {0, 0, 0}, Dp = 0.0;
    double mf = INFINITY, mg = INFINITY;
    int n = 0;
    if (contribs) contribs->clear();
    const std::vector<int32_t> *bin = nullptr;
    if (cx.prefilter) {
        const int bx = std::min(std::max(px / 16, 0), cx.bins_x - 1);
        const int by = std::min(std::max(py / 16, 0), cx.bins_y - 1);
        bin = &cx.bins[size_t(by) * cx.bins_x + bx];
    }
    const size_t count = bin ? bin->size() : cx.order.size();
    for (size_t ii = 0; ii < count; ++ii) {
        const size_t i = bin ? size_t((*bin)[ii]) : ii;
        if (cx.prefilter) {
            const auto &b = cx.box[i];
            if (X < b[0] || X > b[2] || Y < b[1] || Y > b[3]) continue;
        }
        const int64_t k = cx.order[i];
        const Proj &pr = cx.proj[i];
        PairEval e;
        eval_pair(pr, sc.opacities[k], X, Y, e);
        ++*npairs;
        if (!e.hit) continue;
        /* decision margins (R21) */
        const double m_alpha = reldist(e.alpha, kAlphaMin);
        const double m_branch = std::fabs(e.rho_uv - e.rho_lp) / std::max(std::max(e.rho_uv, e.rho_lp), 1e-300);
        mf = std::min(mf, m_alpha);
        mg = std::min(mg, m_alpha);
        if (e.alpha < kAlphaMin) continue;
        mg = std::min(mg, reldist(e.alpha_raw, kAlphaMax));
        mf = std::min(mf, m_branch);
        mg = std::min(mg, m_branch);
        const double tT = T * (1.0 - e.alpha);
        mf = std::min(mf, reldist(tT, kTMin));
        mg = std::min(mg, reldist(tT, kTMin));
        if (tT < kTMin) break;
        const double sg = sc.sigma;
        mg = std::min(mg, std::fabs(std::fabs(e.u) - sg) / sg);
        mg = std::min(mg, std::fabs(std::fabs(e.v) - sg) / sg);
        const int nk = sc.splat_n ? sc.splat_n[k] : N;
        if (nk > 2) {
            const double up = (nk - 1) * (e.u + sg) / (2 * sg), vp = (nk - 1) * (e.v + sg) / (2 * sg);
            if (up > 0 && up < nk - 1) mg = std::min(mg, std::fabs(up - std::round(up)));
            if (vp > 0 && vp < nk - 1) mg = std::min(mg, std::fabs(vp - std::round(vp)));
        }
        Contrib cb;
        cb.k = k;
        cb.e = e;
        cb.T = T;
        bilinear(e.u, e.v, sc.splat_n ? sc.splat_n[k] : N, sg, sc.textures + k * N * N * 3, cb.col, N);
        for (int c = 0; c < 3; ++c) cb.col[c] += pr.rgb_sh[c];
        cb.zi = e.uv_branch ? (pr.T[6] * e.u + pr.T[7] * e.v + pr.T[8]) : pr.T[8];
        const double w = e.alpha * T;
        for (int c = 0; c < 3; ++c) C[c] += cb.col[c] * w;
        Dp += cb.zi * w;
        T = tT;
        ++n;
        if (contribs) contribs->push_back(cb);
    }
    for (int c = 0; c < 3; ++c) rgb[c] = C[c] + T * cx.bg[c];
    *depth = Dp;
    *t_final = T;
    *n_contrib = n;
    *mfwd = mf;
    *mgrad = mg;
}

static int num_threads() {
    const char *e = std::getenv("GBILL_ORACLE_THREADS");
    int n = e ? std::atoi(e) : int(std::thread::hardware_concurrency());
    return n < 1 ? 1 : n;
}

static void build_ctx(Ctx &cx, const orc_scene *sc, const orc_camera *cam, const double *bg,
                      int prefilter) {
    cx.sc = sc;
    cx.cam = cam;
    cx.order = depth_order(*sc, *cam, nullptr);
    cx.proj.resize(cx.order.size());
    cx.box.resize(cx.order.size());
    cx.prefilter = prefilter != 0;
    for (size_t i = 0; i < cx.order.size(); ++i) {
        project(*sc, *cam, cx.order[i], cx.proj[i]);
        if (cx.prefilter) {
            double b[4];
            bbox64(cx.proj[i], 2.0 * std::log(255.0), b);
            /* one pixel of slack on every side */
            cx.box[i] = {b[0] - 1.0, b[1] - 1.0, b[2] + 1.0, b[3] + 1.0};
        }
    }
    for (int c = 0; c < 3; ++c) cx.bg[c] = bg ? bg[c] : 0.0;
    if (cx.prefilter) {
        cx.bins_x = (cam->width + 15) / 16;
        cx.bins_y = (cam->height + 15) / 16;
        cx.bins.assign(size_t(cx.bins_x) * cx.bins_y, {});
        for (size_t i = 0; i < cx.order.size(); ++i) {
            const auto &b = cx.box[i];
            /* pixel centres x + 0.5 inside [b0, b2] */
            const double lx = std::max(std::floor(b[0] - 0.5), 0.0), hx = std::min(std::ceil(b[2] - 0.5), double(cam->width - 1));
            const double ly = std::max(std::floor(b[1] - 0.5), 0.0), hy = std::min(std::ceil(b[3] - 0.5), double(cam->height - 1));
            if (!(lx <= hx) || !(ly <= hy)) continue;
            for (int by = int(ly) / 16; by <= int(hy) / 16; ++by)
                for (int bx = int(lx) / 16; bx <= int(hx) / 16; ++bx)
                    cx.bins[size_t(by) * cx.bins_x + bx].push_back(int32_t(i));
        }
    }
}

int orc_num_threads(void) { return num_threads(); }

int orc_render_forward(const orc_scene *sc, const orc_camera *cam, const orc_window *win,
                       const double *bg, int prefilter, orc_fwd_out *out) {
    Ctx cx;
    build_ctx(cx, sc, cam, bg, prefilter);
    const int nt = std::min(num_threads(), std::max(1, int(win->h)));
    std::vector<int64_t> pairs(nt, 0);
    std::atomic<int> next_row(0);
    auto worker = [&](int tid) {
        for (;;) {
            const int r = next_row.fetch_add(1);
            if (r >= win->h) break;
            for (int c = 0; c < win->w; ++c) {
                const int64_t o = int64_t(r) * win->w + c;
                double rgb[3], depth, tf, mf, mg;
                int nc;
                pixel_forward(cx, win->x0 + c, win->y0 + r, nullptr, rgb, &depth, &tf, &nc, &mf, &mg,
                              &pairs[tid]);
                for (int ch = 0; ch < 3; ++ch) out->rgb[o * 3 + ch] = rgb[ch];
                out->depth[o] = depth;
                out->alpha[o] = 1.0 - tf;
                out->t_final[o] = tf;
                out->n_contrib[o] = nc;
                out->margin_fwd[o] = mf;
                out->margin_grad[o] = mg;
            }
        }
    };
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t) th.emplace_back(worker, t);
    for (auto &t : th) t.join();
    int64_t tot = 0;
    for (auto v : pairs) tot += v;
    if (out->n_pairs) *out->n_pairs = tot;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Backward (Alg. 1 bwd, Alg. 2 adj-bilinear)                               */
/* ------------------------------------------------------------------------ */

/* Per-splat adjoints of the projected quantities, for one view. */
struct SplatAdj {
    double adj_hat[9];  /* d L / d adj(T)        */
    double T_hat[9];    /* d L / d T (direct)    */
    double c_hat[2];    /* d L / d centre        */
    double o_hat;       /* d L / d opacity       */
    double rgb_hat[3];  /* d L / d SH colour     */
};

static void pixel_backward(const Ctx &cx, int px, int py, const std::vector<Contrib> &cb,
                           double t_final, const double dC[3], double dD, double dA,
                           std::vector<SplatAdj> &acc, std::vector<double> &tex_hat,
                           const std::vector<int64_t> &pos_of) {
    const orc_scene &sc = *cx.sc;
    const int N = sc.tex_n;
    const double X = px + 0.5, Y = py + 0.5;
    double S[3] = {0, 0, 0}, SD = 0.0;
    const double bgdot = dC[0] * cx.bg[0] + dC[1] * cx.bg[1] + dC[2] * cx.bg[2];
    for (int i = int(cb.size()) - 1; i >= 0; --i) {
        const Contrib &c = cb[i];
        const PairEval &e = c.e;
        const Proj &pr = cx.proj[pos_of[c.k]];
        SplatAdj &A = acc[pos_of[c.k]];
        const double a = e.alpha, T = c.T, w = a * T;
        /* adjoint of the colour with visibility, then adj-bilinear */
        double chat[3] = {w * dC[0], w * dC[1], w * dC[2]};
        for (int ch = 0; ch < 3; ++ch) A.rgb_hat[ch] += chat[ch];
        double uv_hat[2];
        adj_bilinear(e.u, e.v, sc.splat_n ? sc.splat_n[c.k] : N, sc.sigma, sc.textures + c.k * N * N * 3, chat,
                     tex_hat.data() + c.k * N * N * 3, uv_hat, N);
        double u_hat = uv_hat[0], v_hat = uv_hat[1];
        /* adjoint of alpha */
        const double inv1ma = 1.0 / (1.0 - a);
        double a_hat = 0.0;
        for (int ch = 0; ch < 3; ++ch) a_hat += dC[ch] * (c.col[ch] * T - S[ch] * inv1ma);
        a_hat += dD * (c.zi * T - SD * inv1ma);
        a_hat += (dA - bgdot) * t_final * inv1ma;
        /* depth contribution adjoint */
        const double zi_hat = dD * w;
        for (int ch = 0; ch < 3; ++ch) S[ch] += c.col[ch] * w;
        SD += c.zi * w;
        /* Gaussian opacity adjoint */
        double rho_hat = 0.0;
        if (!e.clamped) {
            A.o_hat += a_hat * e.G;
            rho_hat = -0.5 * a * a_hat;
        }
        if (e.uv_branch) {
            u_hat += 2.0 * e.u * rho_hat;
            v_hat += 2.0 * e.v * rho_hat;
            /* z_i = T20 u + T21 v + T22 */
            A.T_hat[6] += zi_hat * e.u;
            A.T_hat[7] += zi_hat * e.v;
            A.T_hat[8] += zi_hat;
            u_hat += zi_hat * pr.T[6];
            v_hat += zi_hat * pr.T[7];
        } else {
            A.c_hat[0] += rho_hat * kLowPass * -2.0 * e.dx;
            A.c_hat[1] += rho_hat * kLowPass * -2.0 * e.dy;
            A.T_hat[8] += zi_hat;
        }
        /* adjoint of the ray intersection u = zeta_x / zeta_z, v = zeta_y / zeta_z */
        const double iz = 1.0 / e.zeta[2];
        const double zh[3] = {u_hat * iz, v_hat * iz, -(u_hat * e.u + v_hat * e.v) * iz};
        const double Xv[3] = {X, Y, 1.0};
        for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 3; ++q) A.adj_hat[r * 3 + q] += zh[r] * Xv[q];
    }
}

/* Chains the per-view splat adjoints into the parameter gradients. */
static void chain_splat(const orc_scene &sc, const orc_camera &cam, int64_t k, const Proj &pr,
                        const SplatAdj &A, orc_grads *g) {
    double That[9];
    for (int i = 0; i < 9; ++i) That[i] = A.T_hat[i];
    /* adj(T)[i][j] = T[r1][c1] T[r2][c2] - T[r1][c2] T[r2][c1] */
    const double *T = pr.T;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const int r1 = (j + 1) % 3, r2 = (j + 2) % 3, c1 = (i + 1) % 3, c2 = (i + 2) % 3;
            const double h = A.adj_hat[i * 3 + j];
            That[r1 * 3 + c1] += h * T[r2 * 3 + c2];
            That[r2 * 3 + c2] += h * T[r1 * 3 + c1];
            That[r1 * 3 + c2] -= h * T[r2 * 3 + c1];
            That[r2 * 3 + c1] -= h * T[r1 * 3 + c2];
        }
    /* centre c = (T02 / T22, T12 / T22) */
    That[2] += A.c_hat[0] / T[8];
    That[5] += A.c_hat[1] / T[8];
    That[8] -= (A.c_hat[0] * T[2] + A.c_hat[1] * T[5]) / (T[8] * T[8]);
    /* T = K [a' b' p'] with a' = R a, b' = R b, p' = R p + t */
    double colhat[3][3];
    for (int j = 0; j < 3; ++j) {
        colhat[j][0] = cam.fx * That[0 * 3 + j];
        colhat[j][1] = cam.fy * That[1 * 3 + j];
        colhat[j][2] = cam.cx * That[0 * 3 + j] + cam.cy * That[1 * 3 + j] + That[2 * 3 + j];
    }
    const double *W = cam.w2c;
    double world_hat[3][3];
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i)
            world_hat[j][i] = W[0 * 4 + i] * colhat[j][0] + W[1 * 4 + i] * colhat[j][1] + W[2 * 4 + i] * colhat[j][2];
    const double *s = sc.scales + 2 * k;
    double tu_hat[3], tv_hat[3];
    double su_hat = 0, sv_hat = 0;
    for (int i = 0; i < 3; ++i) {
        su_hat += world_hat[0][i] * pr.tu[i];
        sv_hat += world_hat[1][i] * pr.tv[i];
        tu_hat[i] = s[0] * world_hat[0][i];
        tv_hat[i] = s[1] * world_hat[1][i];
    }
    double p_hat[3] = {world_hat[2][0], world_hat[2][1], world_hat[2][2]};
    /* SH colour */
    const int D = sc.sh_degree, M = (D + 1) * (D + 1);
    double Y[16], dY[16][3];
    sh_eval(D, pr.dir, Y, dY);
    const double *kk = sc.sh + k * M * 3;
    double dir_hat[3] = {0, 0, 0};
    for (int m = 0; m < M; ++m)
        for (int c = 0; c < 3; ++c) {
            g->d_sh[(k * M + m) * 3 + c] += Y[m] * A.rgb_hat[c];
            for (int i = 0; i < 3; ++i) dir_hat[i] += kk[m * 3 + c] * A.rgb_hat[c] * dY[m][i];
        }
    const double dd = dir_hat[0] * pr.dir[0] + dir_hat[1] * pr.dir[1] + dir_hat[2] * pr.dir[2];
    for (int i = 0; i < 3; ++i) p_hat[i] += (dir_hat[i] - pr.dir[i] * dd) / pr.dist;
    /* rotation columns -> normalised quaternion -> raw quaternion */
    const double w = pr.qn[0], x = pr.qn[1], y = pr.qn[2], z = pr.qn[3];
    /* t_u = (1-2(y^2+z^2), 2(xy+wz), 2(xz-wy)),  t_v = (2(xy-wz), 1-2(x^2+z^2), 2(yz+wx)) */
    double qh[4];
    qh[0] = tu_hat[1] * 2 * z - tu_hat[2] * 2 * y - tv_hat[0] * 2 * z + tv_hat[2] * 2 * x;
    qh[1] = tu_hat[1] * 2 * y + tu_hat[2] * 2 * z + tv_hat[0] * 2 * y - tv_hat[1] * 4 * x + tv_hat[2] * 2 * w;
    qh[2] = -tu_hat[0] * 4 * y + tu_hat[1] * 2 * x - tu_hat[2] * 2 * w + tv_hat[0] * 2 * x + tv_hat[2] * 2 * z;
    qh[3] = -tu_hat[0] * 4 * z + tu_hat[1] * 2 * w + tu_hat[2] * 2 * x - tv_hat[0] * 2 * w - tv_hat[1] * 4 * z + tv_hat[2] * 2 * y;
    const double qd = qh[0] * w + qh[1] * x + qh[2] * y + qh[3] * z;
    for (int i = 0; i < 4; ++i) g->d_quats[4 * k + i] += (qh[i] - pr.qn[i] * qd) / pr.qnorm;
    g->d_scales[2 * k + 0] += su_hat;
    g->d_scales[2 * k + 1] += sv_hat;
    for (int i = 0; i < 3; ++i) g->d_means[3 * k + i] += p_hat[i];
    g->d_opacities[k] += A.o_hat;
}

int orc_render_backward(const orc_scene *sc, const orc_camera *cam, const orc_window *win,
                        const double *bg, int prefilter, const double *dL_drgb,
                        const double *dL_ddepth, const double *dL_dalpha, orc_grads *g) {
    Ctx cx;
    build_ctx(cx, sc, cam, bg, prefilter);
    std::vector<int64_t> pos_of(sc->num_splats, -1);
    for (size_t i = 0; i < cx.order.size(); ++i) pos_of[cx.order[i]] = int64_t(i);
    const int nt = std::min(num_threads(), std::max(1, int(win->h)));
    const int N = sc->tex_n;
    std::vector<std::vector<SplatAdj>> acc(nt);
    std::vector<std::vector<double>> tex(nt);
    /* fixed row partition: thread t owns rows t, t+nt, ... (deterministic sums) */
    auto worker = [&](int tid) {
        acc[tid].assign(cx.order.size(), SplatAdj{});
        tex[tid].assign(size_t(sc->num_splats) * N * N * 3, 0.0);
        std::vector<Contrib> cb;
        int64_t np = 0;
        for (int r = tid; r < win->h; r += nt)
            for (int c = 0; c < win->w; ++c) {
                const int64_t o = int64_t(r) * win->w + c;
                double rgb[3], depth, tf, mf, mg;
                int nc;
                pixel_forward(cx, win->x0 + c, win->y0 + r, &cb, rgb, &depth, &tf, &nc, &mf, &mg, &np);
                const double dD = dL_ddepth ? dL_ddepth[o] : 0.0;
                const double dA = dL_dalpha ? dL_dalpha[o] : 0.0;
                pixel_backward(cx, win->x0 + c, win->y0 + r, cb, tf, dL_drgb + 3 * o, dD, dA, acc[tid],
                               tex[tid], pos_of);
            }
    };
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t) th.emplace_back(worker, t);
    for (auto &t : th) t.join();
    for (size_t i = 0; i < cx.order.size(); ++i) {
        SplatAdj A{};
        for (int t = 0; t < nt; ++t) {
            const SplatAdj &B = acc[t][i];
            for (int j = 0; j < 9; ++j) { A.adj_hat[j] += B.adj_hat[j]; A.T_hat[j] += B.T_hat[j]; }
            A.c_hat[0] += B.c_hat[0]; A.c_hat[1] += B.c_hat[1];
            A.o_hat += B.o_hat;
            for (int c = 0; c < 3; ++c) A.rgb_hat[c] += B.rgb_hat[c];
        }
        chain_splat(*sc, *cam, cx.order[i], cx.proj[i], A, g);
    }
    const size_t ntex = size_t(sc->num_splats) * N * N * 3;
    for (int t = 0; t < nt; ++t)
        for (size_t j = 0; j < ntex; ++j) g->d_textures[j] += tex[t][j];
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Entry points used by the pins                                            */
/* ------------------------------------------------------------------------ */

/* Contributor list of one pixel: splat id, alpha and transmittance before it. */
int orc_pixel_trace(const orc_scene *sc, const orc_camera *cam, int32_t px, int32_t py, int32_t cap,
                    int64_t *ids, double *alpha, double *trans, double *t_final) {
    Ctx cx;
    build_ctx(cx, sc, cam, nullptr, 0);
    std::vector<Contrib> cb;
    double rgb[3], depth, tf, mf, mg;
    int nc;
    int64_t np = 0;
    pixel_forward(cx, px, py, &cb, rgb, &depth, &tf, &nc, &mf, &mg, &np);
    for (int i = 0; i < nc && i < cap; ++i) {
        ids[i] = cb[i].k;
        alpha[i] = cb[i].e.alpha;
        trans[i] = cb[i].T;
    }
    *t_final = tf;
    return nc;
}

/* FP32 culling, pixel rectangles and depth of every splat in one view. */
int orc_keys32(const orc_scene *sc, const orc_camera *cam, int32_t *valid, float *depth,
               int32_t *prect) {
    for (int64_t k = 0; k < sc->num_splats; ++k) {
        float z = 0.0f;
        int r[4] = {0, 0, -1, -1};
        valid[k] = splat_key(*sc, *cam, k, &z, r);
        depth[k] = z;
        for (int i = 0; i < 4; ++i) prect[4 * k + i] = r[i];
    }
    return 0;
}

/* FP64 projection of every splat in one view (for closed-form pins). */
int orc_project(const orc_scene *sc, const orc_camera *cam, double *T, double *adj, double *centre,
                double *rgb_sh, double *bbox) {
    for (int64_t k = 0; k < sc->num_splats; ++k) {
        Proj pr;
        project(*sc, *cam, k, pr);
        for (int i = 0; i < 9; ++i) { T[9 * k + i] = pr.T[i]; adj[9 * k + i] = pr.adj[i]; }
        centre[2 * k] = pr.c[0];
        centre[2 * k + 1] = pr.c[1];
        for (int c = 0; c < 3; ++c) rgb_sh[3 * k + c] = pr.rgb_sh[c];
        if (bbox) bbox64(pr, 2.0 * std::log(255.0), bbox + 4 * k);
    }
    return 0;
}

/* Per-pair evaluation for one splat over a list of pixel centres. */
int orc_eval_pairs(const orc_scene *sc, const orc_camera *cam, int64_t k, const double *xy, int64_t n,
                   double *u, double *v, double *alpha, int32_t *uv_branch) {
    Proj pr;
    project(*sc, *cam, k, pr);
    for (int64_t i = 0; i < n; ++i) {
        PairEval e;
        eval_pair(pr, sc->opacities[k], xy[2 * i], xy[2 * i + 1], e);
        u[i] = e.hit ? e.u : NAN;
        v[i] = e.hit ? e.v : NAN;
        alpha[i] = e.hit ? e.alpha : 0.0;
        uv_branch[i] = e.hit ? int(e.uv_branch) : -1;
    }
    return 0;
}

int orc_sh_basis(int32_t D, const double *dirs, int64_t n, double *Y, double *dY) {
    const int M = (D + 1) * (D + 1);
    for (int64_t i = 0; i < n; ++i) {
        double y[16], g[16][3];
        sh_eval(D, dirs + 3 * i, y, g);
        for (int m = 0; m < M; ++m) {
            Y[i * M + m] = y[m];
            if (dY)
                for (int j = 0; j < 3; ++j) dY[(i * M + m) * 3 + j] = g[m][j];
        }
    }
    return 0;
}

int orc_bilinear(const double *uv, int64_t n, int32_t N, double sigma, const double *C, double *out) {
    for (int64_t i = 0; i < n; ++i) bilinear(uv[2 * i], uv[2 * i + 1], N, sigma, C, out + 3 * i);
    return 0;
}

int orc_adj_bilinear(const double *uv, int64_t n, int32_t N, double sigma, const double *C,
                     const double *chat, double *Chat, double *uv_hat) {
    for (int64_t i = 0; i < n; ++i)
        adj_bilinear(uv[2 * i], uv[2 * i + 1], N, sigma, C, chat + 3 * i, Chat, uv_hat + 2 * i);
    return 0;
}

} /* extern "C" */
