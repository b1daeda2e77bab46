/*
 * mcdi oracle -- a plain, slow, FP64 CPU restatement of the differentiable
 * Monte Carlo direct-illumination estimator of Hasselgren, Hofmann and
 * Munkberg, "Shape, Light, and Material Decomposition from Images using Monte
 * Carlo Rendering and Denoising" (NeurIPS 2022, arXiv 2206.03380).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The CUDA library never
 * links, includes or calls it, and it shares no code with the CUDA library.
 *
 * Everything is computed in double precision, one pixel and one sample at a
 * time, in the order the paper states the method:
 *   1. counter-based random numbers (Philox4x32-10, Salmon et al. 2011), so
 *      that the forward pass and the adjoint see the same samples (Sec. 4.1,
 *      App. D "correlated samples");
 *   2. the lat-long light probe and its piecewise-constant 2D sampling
 *      distribution (Sec. 3 "HDR light probe", Sec. 4.1, App. D);
 *   3. cosine-weighted hemisphere sampling for the diffuse lobe (Sec. 4.1);
 *   4. the GGX lobe: normal distribution, Smith masking, visible-normal
 *      sampling (Heitz 2018, cited in Sec. 4.1) and Schlick Fresnel;
 *   5. shadow-ray visibility by brute force over every triangle (Sec. 3.1,
 *      with the leakage term H = 1 - tau of App. A);
 *   6. the primary-visibility G-buffer by brute-force closest hit;
 *   7. the MIS estimator with the balance heuristic (Sec. 4.1, Eq. of the
 *      MIS estimator) split into demodulated diffuse c_d, reflectance k_d and
 *      specular c_s (Sec. 4.2, light separation);
 *   8. the frozen-sample estimator (detached sampling, Sec. 4.1; detached
 *      shadow visibility, Sec. 3.1 "Shadow gradients") and its analytic
 *      adjoint;
 *   9. the shadow-visibility gradient the paper evaluates as an ablation
 *      (appendix "Visibility gradients from shadows"): the boundary term of
 *      the blocked set, estimated by edge sampling over the mesh's edge table.
 *
 * Where the paper is silent the reading taken is stated at the function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* 0. small vector helpers                                                   */
/* ------------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double a[3], const double b[3], double o[3]) {
    double x = a[1] * b[2] - a[2] * b[1];
    double y = a[2] * b[0] - a[0] * b[2];
    double z = a[0] * b[1] - a[1] * b[0];
    o[0] = x; o[1] = y; o[2] = z;
}
static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }
static void normalize3(double a[3]) {
    double l = norm3(a);
    a[0] /= l; a[1] /= l; a[2] /= l;
}
static void sub3(const double a[3], const double b[3], double o[3]) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }

/* ------------------------------------------------------------------------ */
/* 1. Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC 2011)                 */
/*    One round maps (c0,c1,c2,c3) with key (k0,k1) to                        */
/*      (hi(B*c2) ^ c1 ^ k0, lo(B*c2), hi(A*c0) ^ c3 ^ k1, lo(A*c0))          */
/*    with multipliers A = 0xD2511F53, B = 0xCD9E8D57; between rounds the key */
/*    is bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85).               */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t pa = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t pb = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(pb >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)pb;
        uint32_t n2 = (uint32_t)(pa >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)pa;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The two uniforms of one sample.  Counter = (pixel, view, sample, stream),
 * key = (seed low word, seed high word).  A 32-bit output x becomes
 * (x >> 8) * 2^-24, a 24-bit fraction that is exact in float and double, so
 * both implementations see the very same number in [0, 1). */
void orc_sample_uniforms(uint64_t seed, uint32_t pixel, uint32_t view, uint32_t sample, uint32_t stream,
                         double u[2]) {
    uint32_t ctr[4] = {pixel, view, sample, stream};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    u[0] = (double)(x[0] >> 8) * (1.0 / 16777216.0);
    u[1] = (double)(x[1] >> 8) * (1.0 / 16777216.0);
}

/* ------------------------------------------------------------------------ */
/* 2. The light probe (Sec. 3: HDR probe stored as a float texture).          */
/*    Reading: lat-long, y up.  (u,v) in [0,1)^2 maps to phi = 2 pi u,        */
/*    theta = pi v and omega = (sin t cos p, cos t, sin t sin p).  Texel       */
/*    (i,j) covers u in [i/W,(i+1)/W), v in [j/H,(j+1)/H); radiance lookup is  */
/*    nearest-texel, i.e. piecewise constant like the sampling density.       */
/* ------------------------------------------------------------------------ */
void orc_dir_from_uv(double u, double v, double d[3]) {
    double phi = 2.0 * ORC_PI * u, theta = ORC_PI * v;
    d[0] = sin(theta) * cos(phi);
    d[1] = cos(theta);
    d[2] = sin(theta) * sin(phi);
}

void orc_uv_from_dir(const double d[3], double* u, double* v) {
    double y = d[1] < -1.0 ? -1.0 : (d[1] > 1.0 ? 1.0 : d[1]);
    *v = acos(y) / ORC_PI;
    double uu = atan2(d[2], d[0]) / (2.0 * ORC_PI);
    if (uu < 0.0) uu += 1.0;
    *u = uu;
}

/* texel index j*W + i of a direction; also reports the distance (in texel
 * units) from the direction's (u,v) to the nearest texel border */
int orc_texel_of_dir(const double d[3], int W, int H, double* border_dist) {
    double u, v;
    orc_uv_from_dir(d, &u, &v);
    double x = u * W, y = v * H;
    int i = (int)floor(x), j = (int)floor(y);
    if (i < 0) i = 0;
    if (i > W - 1) i = W - 1;
    if (j < 0) j = 0;
    if (j > H - 1) j = H - 1;
    if (border_dist) {
        double fx = x - floor(x), fy = y - floor(y);
        double m = fx < 1.0 - fx ? fx : 1.0 - fx;
        double my = fy < 1.0 - fy ? fy : 1.0 - fy;
        *border_dist = m < my ? m : my;
    }
    return j * W + i;
}

/* ------------------------------------------------------------------------ */
/* 3. Piecewise-constant 2D distribution over the probe (Sec. 4.1 "light     */
/*    importance sampling ... piecewise-constant 2D distribution"; App. D;    */
/*    rebuilt whenever the probe changes, Sec. 4.1).                          */
/*    Reading: texel weight w_ij = max(Y,0) * sin(theta_j), Y = (r+g+b)/3 the */
/*    paper's luminance operator (App. A, light regulariser) and theta_j the   */
/*    texel-centre polar angle (the sin accounts for the lat-long area).       */
/*    cond[j][k] = sum_{i<k} w_ij / R_j with cond[j][W] = 1; a row with R_j=0 */
/*    gets the uniform cdf k/W.  marg[k] = sum_{j<k} R_j / T, marg[H] = 1;    */
/*    T = 0 gives the uniform k/H (and the light technique is switched off).  */
/* ------------------------------------------------------------------------ */
void orc_envmap_cdf(const float* env, int W, int H, double* cond, double* marg, double* row_sum, double* total) {
    double T = 0.0;
    for (int j = 0; j < H; ++j) {
        double s = sin(ORC_PI * (j + 0.5) / H);
        double R = 0.0;
        double* c = cond + (size_t)j * (W + 1);
        for (int i = 0; i < W; ++i) {
            const float* t = env + 4 * ((size_t)j * W + i);
            double Y = ((double)t[0] + (double)t[1] + (double)t[2]) / 3.0;
            if (Y < 0.0) Y = 0.0;
            c[i] = R; /* running sum before texel i */
            R += Y * s;
        }
        for (int i = 0; i < W; ++i) c[i] = R > 0.0 ? c[i] / R : (double)i / W;
        c[W] = 1.0;
        row_sum[j] = R;
        marg[j] = T;
        T += R;
    }
    for (int j = 0; j < H; ++j) marg[j] = T > 0.0 ? marg[j] / T : (double)j / H;
    marg[H] = 1.0;
    *total = T;
}

/* largest k in [0, n-1] with cdf[k] <= u (cdf[0] = 0 <= u always) */
static int upper_index(const float* cdf, int n, double u) {
    int k = 0;
    for (int i = 0; i < n; ++i)
        if ((double)cdf[i] <= u) k = i;
    return k;
}

/* Sampling runs on the float tables: they define the distribution, so the
 * density below is the exact density of the sampled points.
 * pdf over (u,v):   W*H*(marg[j+1]-marg[j])*(cond[j][i+1]-cond[j][i])
 * pdf over omega:   pdf_uv / (2 pi^2 sin theta)   (d omega = 2 pi^2 sin t du dv)
 * Returns 0 (no sample) when the probe is black. */
int orc_sample_light(const float* cond32, const float* marg32, int W, int H, double total, double u0, double u1,
                     double d[3], int* texel, double* pdf, double* search_margin) {
    if (!(total > 0.0)) return 0;
    int j = upper_index(marg32, H, u0);
    double wr = (double)marg32[j + 1] - (double)marg32[j];
    double dv = (u0 - marg32[j]) / wr;
    const float* c = cond32 + (size_t)j * (W + 1);
    int i = upper_index(c, W, u1);
    double wc = (double)c[i + 1] - (double)c[i];
    double du = (u1 - c[i]) / wc;
    double u = (i + du) / W, v = (j + dv) / H;
    orc_dir_from_uv(u, v, d);
    *texel = j * W + i;
    double st = sin(ORC_PI * v);
    *pdf = st > 0.0 ? (W * (double)H * wr * wc) / (2.0 * ORC_PI * ORC_PI * st) : 0.0;
    if (search_margin) {
        /* how close u0/u1 came to a table entry (a tie a 1-ulp table difference could flip) */
        double m = fabs(u0 - marg32[j]);
        if (fabs(marg32[j + 1] - u0) < m) m = fabs(marg32[j + 1] - u0);
        if (fabs(u1 - c[i]) < m) m = fabs(u1 - c[i]);
        if (fabs(c[i + 1] - u1) < m) m = fabs(c[i + 1] - u1);
        *search_margin = m;
    }
    return 1;
}

double orc_pdf_light(const float* cond32, const float* marg32, int W, int H, double total, const double d[3]) {
    if (!(total > 0.0)) return 0.0;
    int t = orc_texel_of_dir(d, W, H, NULL);
    int j = t / W, i = t % W;
    double wr = (double)marg32[j + 1] - (double)marg32[j];
    double wc = (double)cond32[(size_t)j * (W + 1) + i + 1] - (double)cond32[(size_t)j * (W + 1) + i];
    double y = d[1];
    double st2 = 1.0 - y * y;
    double st = st2 > 0.0 ? sqrt(st2) : 0.0;
    return st > 0.0 ? (W * (double)H * wr * wc) / (2.0 * ORC_PI * ORC_PI * st) : 0.0;
}

/* ------------------------------------------------------------------------ */
/* 4. Cosine-weighted hemisphere sampling for the diffuse lobe (Sec. 4.1).  */
/*    Reading: polar map r = sqrt(u0), phi = 2 pi u1, lifted to the           */
/*    hemisphere; tangent frame of Duff et al. 2017 with sign(0) = +1.        */
/* ------------------------------------------------------------------------ */
void orc_frame(const double n[3], double b1[3], double b2[3]) {
    double s = n[2] >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (s + n[2]);
    double b = n[0] * n[1] * a;
    b1[0] = 1.0 + s * n[0] * n[0] * a; b1[1] = s * b; b1[2] = -s * n[0];
    b2[0] = b; b2[1] = s + n[1] * n[1] * a; b2[2] = -n[1];
}

static void to_world(const double n[3], const double l[3], double w[3]) {
    double b1[3], b2[3];
    orc_frame(n, b1, b2);
    for (int k = 0; k < 3; ++k) w[k] = l[0] * b1[k] + l[1] * b2[k] + l[2] * n[k];
}

void orc_sample_cosine(const double n[3], double u0, double u1, double d[3]) {
    double r = sqrt(u0), phi = 2.0 * ORC_PI * u1;
    double l[3] = {r * cos(phi), r * sin(phi), sqrt(1.0 - u0)};
    to_world(n, l, d);
}

double orc_pdf_cosine(const double n[3], const double d[3]) {
    double c = dot3(n, d);
    return c > 0.0 ? c / ORC_PI : 0.0;
}

/* ------------------------------------------------------------------------ */
/* 5. The specular GGX lobe (Sec. 3: Disney PBR = diffuse + isotropic GGX,   */
/*    Walter et al. 2007).  Reading: alpha = max(r^2, 1e-4); D is the GGX      */
/*    (Trowbridge-Reitz) distribution, masking is Smith's with the GGX Lambda  */
/*    and the height-correlated form G2 = 1/(1+Lambda_o+Lambda_i); Fresnel is  */
/*    Schlick's with F0 = 0.04(1-m) + k_d m.                                   */
/* ------------------------------------------------------------------------ */
double orc_alpha(double r) {
    double a = r * r;
    return a > 1e-4 ? a : 1e-4;
}

double orc_ggx_D(double nh, double alpha) {
    if (!(nh > 0.0)) return 0.0;
    double a2 = alpha * alpha;
    double d = nh * nh * (a2 - 1.0) + 1.0;
    return a2 / (ORC_PI * d * d);
}

/* Lambda(c) for a direction with cosine c to the normal */
double orc_ggx_lambda(double c, double alpha) {
    double z = alpha * alpha * (1.0 / (c * c) - 1.0);
    return 0.5 * (sqrt(1.0 + z) - 1.0);
}

double orc_ggx_G1(double c, double alpha) { return 1.0 / (1.0 + orc_ggx_lambda(c, alpha)); }

double orc_ggx_G2(double ci, double co, double alpha) {
    return 1.0 / (1.0 + orc_ggx_lambda(ci, alpha) + orc_ggx_lambda(co, alpha));
}

double orc_schlick(double f0, double vh) {
    double x = 1.0 - (vh < 0.0 ? 0.0 : (vh > 1.0 ? 1.0 : vh));
    return f0 + (1.0 - f0) * x * x * x * x * x;
}

/* Visible-normal sampling (Heitz 2018, "Sampling the GGX distribution of
 * visible normals"): stretch the view to the unit-roughness configuration,
 * sample the projected hemisphere with the half-disk warp, unstretch.  The
 * light direction is the view mirrored about the sampled micro-normal.
 * wo_local = view in the (b1, b2, n) frame, wo_local[2] > 0. */
void orc_sample_vndf_local(const double wo[3], double alpha, double u0, double u1, double h[3]) {
    double vh[3] = {alpha * wo[0], alpha * wo[1], wo[2]};
    normalize3(vh);
    double lensq = vh[0] * vh[0] + vh[1] * vh[1];
    double t1v[3], t2v[3];
    if (lensq > 0.0) {
        double il = 1.0 / sqrt(lensq);
        t1v[0] = -vh[1] * il; t1v[1] = vh[0] * il; t1v[2] = 0.0;
    } else {
        t1v[0] = 1.0; t1v[1] = 0.0; t1v[2] = 0.0;
    }
    cross3(vh, t1v, t2v);
    double r = sqrt(u0), phi = 2.0 * ORC_PI * u1;
    double t1 = r * cos(phi), t2 = r * sin(phi);
    double s = 0.5 * (1.0 + vh[2]);
    t2 = (1.0 - s) * sqrt(1.0 - t1 * t1) + s * t2;
    double tz = 1.0 - t1 * t1 - t2 * t2;
    tz = tz > 0.0 ? sqrt(tz) : 0.0;
    double nh[3];
    for (int k = 0; k < 3; ++k) nh[k] = t1 * t1v[k] + t2 * t2v[k] + tz * vh[k];
    h[0] = alpha * nh[0];
    h[1] = alpha * nh[1];
    h[2] = nh[2] > 0.0 ? nh[2] : 0.0;
    normalize3(h);
}

/* world-space GGX sample for shading normal n and view wo (co = n.wo > 0) */
void orc_sample_ggx(const double n[3], const double wo[3], double alpha, double u0, double u1, double d[3]) {
    double b1[3], b2[3];
    orc_frame(n, b1, b2);
    double lo[3] = {dot3(wo, b1), dot3(wo, b2), dot3(wo, n)};
    double hl[3], h[3];
    orc_sample_vndf_local(lo, alpha, u0, u1, hl);
    to_world(n, hl, h);
    double vh = dot3(wo, h);
    for (int k = 0; k < 3; ++k) d[k] = 2.0 * vh * h[k] - wo[k];
}

/* density of the GGX technique over light directions:
 * VNDF  D_wo(h) = G1(wo) max(0, wo.h) D(h) / (n.wo), times the reflection
 * Jacobian 1/(4 wo.h) = G1(wo) D(h) / (4 n.wo). */
double orc_pdf_ggx(const double n[3], const double wo[3], double alpha, const double d[3]) {
    double co = dot3(n, wo);
    double h[3] = {d[0] + wo[0], d[1] + wo[1], d[2] + wo[2]};
    double l = norm3(h);
    if (!(l > 0.0)) return 0.0;
    h[0] /= l; h[1] /= l; h[2] /= l;
    if (!(dot3(wo, h) > 0.0)) return 0.0;
    return orc_ggx_G1(co, alpha) * orc_ggx_D(dot3(n, h), alpha) / (4.0 * co);
}

/* ------------------------------------------------------------------------ */
/* 6. Ray/triangle visibility (Sec. 3.1: L_i includes a visibility test by a  */
/*    shadow ray).  Moller-Trumbore, two-sided, edges inclusive, t > 0.       */
/* ------------------------------------------------------------------------ */
/* returns 1 on a hit (t > 0); t,u,v are written when the ray meets the plane */
int orc_ray_triangle(const double o[3], const double d[3], const double v0[3], const double v1[3],
                     const double v2[3], double* t, double* u, double* v) {
    double e1[3], e2[3], p[3], s[3], q[3];
    sub3(v1, v0, e1);
    sub3(v2, v0, e2);
    cross3(d, e2, p);
    double det = dot3(e1, p);
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    sub3(o, v0, s);
    *u = dot3(s, p) * inv;
    cross3(s, e1, q);
    *v = dot3(d, q) * inv;
    *t = dot3(e2, q) * inv;
    if (*u < 0.0 || *v < 0.0 || *u + *v > 1.0) return 0;
    return *t > 0.0;
}

static void load_vert(const float* verts, int idx, double o[3]) {
    o[0] = verts[3 * (size_t)idx]; o[1] = verts[3 * (size_t)idx + 1]; o[2] = verts[3 * (size_t)idx + 2];
}

/* any-hit by brute force over every triangle.  With margin != NULL it scans
 * them all and reports min |min(u, v, 1-u-v)| over triangles whose plane the
 * ray crosses at t > 0 (how close the decision came to an edge), and the
 * smallest |t| of such a crossing within the triangle bounds. */
int orc_any_hit(const float* verts, const int* tris, int n_tris, const double o[3], const double d[3],
                double* edge_margin, double* t_margin) {
    int hit = 0;
    double em = INFINITY, tm = INFINITY;
    for (int k = 0; k < n_tris; ++k) {
        double a[3], b[3], c[3], t, u, v;
        load_vert(verts, tris[3 * k], a);
        load_vert(verts, tris[3 * k + 1], b);
        load_vert(verts, tris[3 * k + 2], c);
        int h = orc_ray_triangle(o, d, a, b, c, &t, &u, &v);
        if (h) hit = 1;
        if (!edge_margin) {
            if (hit) return 1;
            continue;
        }
        /* recompute the plane crossing for the margin (also for misses) */
        double e1[3], e2[3], p[3], s[3], q[3];
        sub3(b, a, e1);
        sub3(c, a, e2);
        cross3(d, e2, p);
        double det = dot3(e1, p);
        if (det == 0.0) continue;
        sub3(o, a, s);
        cross3(s, e1, q);
        double uu = dot3(s, p) / det, vv = dot3(d, q) / det, tt = dot3(e2, q) / det;
        double bm = uu;
        if (vv < bm) bm = vv;
        if (1.0 - uu - vv < bm) bm = 1.0 - uu - vv;
        if (tt > 0.0 && fabs(bm) < em) em = fabs(bm);
        if (bm >= 0.0 && fabs(tt) < tm) tm = fabs(tt);
    }
    if (edge_margin) *edge_margin = em;
    if (t_margin) *t_margin = tm;
    return hit;
}

/* closest hit by brute force; returns the triangle index or -1 */
int orc_closest_hit(const float* verts, const int* tris, int n_tris, const double o[3], const double d[3],
                    double* t_out, double* u_out, double* v_out) {
    int best = -1;
    double bt = INFINITY;
    for (int k = 0; k < n_tris; ++k) {
        double a[3], b[3], c[3], t, u, v;
        load_vert(verts, tris[3 * k], a);
        load_vert(verts, tris[3 * k + 1], b);
        load_vert(verts, tris[3 * k + 2], c);
        if (orc_ray_triangle(o, d, a, b, c, &t, &u, &v) && t < bt) {
            bt = t;
            best = k;
            *u_out = u;
            *v_out = v;
        }
    }
    *t_out = bt;
    return best;
}

/* ------------------------------------------------------------------------ */
/* 7. Primary visibility: the G-buffer (the paper rasterizes it with          */
/*    nvdiffrast, Sec. 3 and 3.1; here a pinhole closest-hit ray cast stands  */
/*    in).  cam = {origin[3], right[3], up[3], forward[3], tan(fovy/2),       */
/*    aspect}.  Pixel (x,y), y down:                                           */
/*      dir = normalize(fwd + sx right + sy up),                               */
/*      sx = (2(x+.5)/W - 1) tan aspect,  sy = (1 - 2(y+.5)/H) tan.           */
/*    Position and normal are barycentric interpolations of the vertices and  */
/*    vertex normals; k_d and k_orm are bilinear (clamp-to-edge) lookups of   */
/*    T x T float4 textures at the planar coordinate                          */
/*    ((x - ox) s, (z - oz) s).  A miss writes zeros (coverage 0).            */
/* ------------------------------------------------------------------------ */
void orc_camera_ray(const double cam[14], int Wpx, int Hpx, int x, int y, double d[3]) {
    double sx = (2.0 * (x + 0.5) / Wpx - 1.0) * cam[12] * cam[13];
    double sy = (1.0 - 2.0 * (y + 0.5) / Hpx) * cam[12];
    for (int k = 0; k < 3; ++k) d[k] = cam[9 + k] + sx * cam[3 + k] + sy * cam[6 + k];
    normalize3(d);
}

void orc_texture_bilinear(const float* tex, int T, double u, double v, double out[4]) {
    double x = u * T - 0.5, y = v * T - 0.5;
    double x0 = floor(x), y0 = floor(y);
    double fx = x - x0, fy = y - y0;
    int xi[2] = {(int)x0, (int)x0 + 1}, yi[2] = {(int)y0, (int)y0 + 1};
    for (int k = 0; k < 2; ++k) {
        if (xi[k] < 0) xi[k] = 0;
        if (xi[k] > T - 1) xi[k] = T - 1;
        if (yi[k] < 0) yi[k] = 0;
        if (yi[k] > T - 1) yi[k] = T - 1;
    }
    for (int c = 0; c < 4; ++c) {
        double t00 = tex[4 * ((size_t)yi[0] * T + xi[0]) + c], t10 = tex[4 * ((size_t)yi[0] * T + xi[1]) + c];
        double t01 = tex[4 * ((size_t)yi[1] * T + xi[0]) + c], t11 = tex[4 * ((size_t)yi[1] * T + xi[1]) + c];
        double top = t00 + (t10 - t00) * fx, bot = t01 + (t11 - t01) * fx;
        out[c] = top + (bot - top) * fy;
    }
}

/* G-buffer rows for a list of pixels (y*W + x); each row is 16 doubles:
 * pos.xyz coverage | normal.xyz 0 | k_d.rgb 0 | k_orm.(o,r,m) 0 */
void orc_primary_cast(const float* verts, const float* vnrm, const int* tris, int n_tris, const double cam[14],
                      int Wpx, int Hpx, const int* pix, int n_pix, const float* tex_kd, const float* tex_korm,
                      int tex_size, const double uvmap[3], double* gb) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int q = 0; q < n_pix; ++q) {
        double* row = gb + 16 * (size_t)q;
        memset(row, 0, 16 * sizeof(double));
        int x = pix[q] % Wpx, y = pix[q] / Wpx;
        double d[3], t, u, v;
        orc_camera_ray(cam, Wpx, Hpx, x, y, d);
        int k = orc_closest_hit(verts, tris, n_tris, cam, d, &t, &u, &v);
        if (k < 0) continue;
        double w = 1.0 - u - v;
        for (int c = 0; c < 3; ++c) {
            row[c] = w * verts[3 * (size_t)tris[3 * k] + c] + u * verts[3 * (size_t)tris[3 * k + 1] + c] +
                     v * verts[3 * (size_t)tris[3 * k + 2] + c];
            row[4 + c] = w * vnrm[3 * (size_t)tris[3 * k] + c] + u * vnrm[3 * (size_t)tris[3 * k + 1] + c] +
                         v * vnrm[3 * (size_t)tris[3 * k + 2] + c];
        }
        row[3] = 1.0;
        double tu = (row[0] - uvmap[0]) * uvmap[2], tv = (row[2] - uvmap[1]) * uvmap[2];
        double kd[4], korm[4];
        orc_texture_bilinear(tex_kd, tex_size, tu, tv, kd);
        orc_texture_bilinear(tex_korm, tex_size, tu, tv, korm);
        for (int c = 0; c < 3; ++c) {
            row[8 + c] = kd[c];
            row[12 + c] = korm[c];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* 8. The MIS direct-illumination estimator (Sec. 3.1 MC estimator; Sec. 4.1 */
/*    MIS with the balance heuristic; Sec. 4.2 light separation).            */
/*                                                                            */
/*    With n_k samples of technique k, the balance-heuristic estimator         */
/*       sum_k (1/n_k) sum_j w_k g/p_k,  w_k = n_k p_k / sum_l n_l p_l         */
/*    reduces to  sum over all samples of  g(w) / sum_l n_l p_l(w).            */
/*    Techniques: light (piecewise-constant probe), cosine, GGX (VNDF).       */
/*    Sample j < n_L is a light sample, then n_C cosine, then n_G GGX.        */
/*    g(w) = L(w) H(w) f(w, wo) (n.w)^+  split into                           */
/*      c_d += L H (n.w) / pi           (demodulated diffuse)                  */
/*      c_s += L H D G2 F / (4 n.wo)    (specular, = L H f_s (n.w))            */
/*    and k_d,out = k_d (1 - m).                                               */
/*    Readings: the lobe is off (f_s = 0, p_ggx = 0) where n.wo < 1e-4; a     */
/*    sample with n.w <= 0 contributes 0 and traces no ray; the shadow ray    */
/*    starts at p + eps n and has no far limit; H = 1 - tau on a hit (App. A */
/*    light leakage); pixels with zero coverage output zeros.                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    double wi[3];      /* sampled light direction (frozen)                  */
    double inv_denom;  /* 1 / sum_k n_k p_k(wi) (frozen), 0 if inactive     */
    double vis;        /* H (frozen)                                        */
    double margin;     /* distance to the nearest discrete decision         */
    int texel;         /* probe texel j*W + i                                */
    int active;        /* contributes: n.wi > 0 and denominator > 0          */
    int technique;     /* 0 light, 1 cosine, 2 GGX                           */
    int occluded;      /* the shadow ray hit                                  */
} orc_sample_rec;

typedef struct {
    int n_light, n_cos, n_ggx;
    uint32_t stream;
    uint64_t seed;
    double tau, ray_eps;
    int want_margin;
} orc_params;

/* gb: n_pix rows of 16 floats (pos4 nrm4 kd4 korm4), cam_pos: 3 per row,
 * ctr: 2 per row (pixel index within its view, view index).
 * out: 12 per row (c_d.rgb, k_d,out.rgb, c_s.rgb, spec_on, coverage, unused),
 * vis: ceil(spp/32) words per row, bit j set when sample j's ray hit,
 * recs: spp per row (may be NULL). */
void orc_shade_fwd(const float* verts, const int* tris, int n_tris, const float* env, int W, int H,
                   const float* cond32, const float* marg32, double total, const float* gb, const double* cam_pos,
                   const uint32_t* ctr, int n_pix, orc_params prm, double* out, uint32_t* vis,
                   orc_sample_rec* recs) {
    const int spp = prm.n_light + prm.n_cos + prm.n_ggx;
    const int nwords = (spp + 31) / 32;
#pragma omp parallel for schedule(dynamic, 4)
    for (int q = 0; q < n_pix; ++q) {
        const float* g = gb + 16 * (size_t)q;
        double* o = out + 12 * (size_t)q;
        memset(o, 0, 12 * sizeof(double));
        uint32_t* vw = vis ? vis + (size_t)q * nwords : NULL;
        if (vw) memset(vw, 0, nwords * sizeof(uint32_t));
        orc_sample_rec* rq = recs ? recs + (size_t)q * spp : NULL;
        if (rq) memset(rq, 0, spp * sizeof(orc_sample_rec));
        double N[3] = {g[4], g[5], g[6]};
        double lN = norm3(N);
        if (!(g[3] > 0.0) || !(lN > 0.0)) continue; /* background */
        double p[3] = {g[0], g[1], g[2]};
        double n[3] = {N[0] / lN, N[1] / lN, N[2] / lN};
        double kd[3] = {g[8], g[9], g[10]};
        double r = g[13], m = g[14];
        double alpha = orc_alpha(r);
        double wo[3];
        sub3(cam_pos + 3 * (size_t)q, p, wo);
        normalize3(wo);
        double co = dot3(n, wo);
        int spec_on = co >= 1e-4;
        double F0[3];
        for (int c = 0; c < 3; ++c) {
            F0[c] = 0.04 * (1.0 - m) + kd[c] * m;
            o[3 + c] = kd[c] * (1.0 - m);
        }
        o[9] = spec_on;
        o[10] = 1.0;
        double nL = prm.n_light, nC = prm.n_cos, nG = spec_on ? prm.n_ggx : 0;
        for (int j = 0; j < spp; ++j) {
            double u[2], wi[3];
            orc_sample_uniforms(prm.seed, ctr[2 * q], ctr[2 * q + 1], (uint32_t)j, prm.stream, u);
            int tech = j < prm.n_light ? 0 : (j < prm.n_light + prm.n_cos ? 1 : 2);
            int texel = -1, ok = 1;
            double margin = INFINITY, plight = 0.0, bd;
            if (tech == 0) {
                double sm;
                ok = orc_sample_light(cond32, marg32, W, H, total, u[0], u[1], wi, &texel, &plight, &sm);
                if (ok) margin = sm;
            } else if (tech == 1) {
                orc_sample_cosine(n, u[0], u[1], wi);
            } else {
                if (spec_on)
                    orc_sample_ggx(n, wo, alpha, u[0], u[1], wi);
                else
                    ok = 0;
            }
            if (rq) {
                rq[j].technique = tech;
                rq[j].texel = -1;
            }
            if (!ok) continue;
            double ci = dot3(n, wi);
            if (fabs(ci) < margin) margin = fabs(ci);
            if (!(ci > 0.0)) {
                if (rq) rq[j].margin = margin;
                continue;
            }
            if (tech != 0) {
                texel = orc_texel_of_dir(wi, W, H, &bd);
                if (bd < margin) margin = bd;
                plight = orc_pdf_light(cond32, marg32, W, H, total, wi);
            }
            double denom = nL * plight + nC * orc_pdf_cosine(n, wi) + (nG > 0 ? nG * orc_pdf_ggx(n, wo, alpha, wi) : 0.0);
            if (!(denom > 0.0)) continue;
            /* shadow ray */
            double so[3] = {p[0] + prm.ray_eps * n[0], p[1] + prm.ray_eps * n[1], p[2] + prm.ray_eps * n[2]};
            double em, tm;
            int hit = orc_any_hit(verts, tris, n_tris, so, wi, prm.want_margin ? &em : NULL,
                                  prm.want_margin ? &tm : NULL);
            if (prm.want_margin) {
                if (em < margin) margin = em;
                if (tm < margin) margin = tm;
            }
            double Hv = hit ? 1.0 - prm.tau : 1.0;
            if (hit && vw) vw[j >> 5] |= 1u << (j & 31);
            const float* L = env + 4 * (size_t)texel;
            double a = Hv / denom;
            for (int c = 0; c < 3; ++c) o[c] += L[c] * a * ci / ORC_PI;
            if (spec_on) {
                double h[3] = {wi[0] + wo[0], wi[1] + wo[1], wi[2] + wo[2]};
                normalize3(h);
                double D = orc_ggx_D(dot3(n, h), alpha);
                double G2 = orc_ggx_G2(ci, co, alpha);
                double vh = dot3(wo, h);
                for (int c = 0; c < 3; ++c) o[6 + c] += L[c] * a * D * G2 * orc_schlick(F0[c], vh) / (4.0 * co);
            }
            if (rq) {
                rq[j].wi[0] = wi[0]; rq[j].wi[1] = wi[1]; rq[j].wi[2] = wi[2];
                rq[j].inv_denom = 1.0 / denom;
                rq[j].vis = Hv;
                rq[j].texel = texel;
                rq[j].active = 1;
                rq[j].occluded = hit;
            }
            if (rq) rq[j].margin = margin;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* 9. Frozen-sample estimator and its adjoint.                               */
/*    Detached sampling (Sec. 4.1, following Zeltner et al.): directions and */
/*    MIS denominators do not move with the parameters; detached shadow      */
/*    visibility (Sec. 3.1 "Shadow gradients"): H does not move either.  The */
/*    function differentiated is therefore, per pixel,                        */
/*      c_d = sum_j a_j L_tj (n.w_j)/pi,                                       */
/*      c_s = sum_j a_j L_tj D(n.h_j) G2(n.w_j, n.wo) F(wo.h_j) / (4 n.wo),    */
/*      k_d,out = k_d (1 - m),                                                 */
/*    a_j = H_j / denominator_j, n = N/|N|, alpha = max(r^2, 1e-4),           */
/*    over the samples active at the frozen point, with the specular lobe     */
/*    switch (n.wo >= 1e-4) frozen too.  Parameters: N, k_d, k_orm = (o,r,m) */
/*    per pixel and the probe texels.  The roughness and metallic grads come  */
/*    only from the specular term and k_d,out; o has no effect.               */
/*    param rows: 12 doubles per pixel: N.xyz, k_d.rgb, (o, r, m), pos.xyz;   */
/*    env3: 3 doubles per texel.                                               */
/* ------------------------------------------------------------------------ */
void orc_frozen_eval(const orc_sample_rec* recs, int spp, int n_pix, const double* prow, const double* cam_pos,
                     const int* spec_on, const double* env3, double* out /* 9 per pixel */) {
#pragma omp parallel for schedule(static)
    for (int q = 0; q < n_pix; ++q) {
        const double* P = prow + 12 * (size_t)q;
        double* o = out + 9 * (size_t)q;
        memset(o, 0, 9 * sizeof(double));
        double N[3] = {P[0], P[1], P[2]};
        double lN = norm3(N);
        if (!(lN > 0.0)) continue;
        double n[3] = {N[0] / lN, N[1] / lN, N[2] / lN};
        const double* kd = P + 3;
        double r = P[7], m = P[8];
        double alpha = orc_alpha(r);
        double wo[3];
        sub3(cam_pos + 3 * (size_t)q, P + 9, wo);
        normalize3(wo);
        double co = dot3(n, wo);
        for (int c = 0; c < 3; ++c) o[3 + c] = kd[c] * (1.0 - m);
        for (int j = 0; j < spp; ++j) {
            const orc_sample_rec* s = recs + (size_t)q * spp + j;
            if (!s->active) continue;
            double a = s->vis * s->inv_denom;
            double ci = dot3(n, s->wi);
            const double* L = env3 + 3 * (size_t)s->texel;
            for (int c = 0; c < 3; ++c) o[c] += a * L[c] * ci / ORC_PI;
            if (spec_on[q]) {
                double h[3] = {s->wi[0] + wo[0], s->wi[1] + wo[1], s->wi[2] + wo[2]};
                normalize3(h);
                double D = orc_ggx_D(dot3(n, h), alpha);
                double G2 = orc_ggx_G2(ci, co, alpha);
                double vh = dot3(wo, h);
                for (int c = 0; c < 3; ++c) {
                    double F0 = 0.04 * (1.0 - m) + kd[c] * m;
                    o[6 + c] += a * L[c] * D * G2 * orc_schlick(F0, vh) / (4.0 * co);
                }
            }
        }
    }
}

/* Per-pixel constants of the frozen estimator's adjoint. */
typedef struct {
    double n[3], wo[3], lN, co, alpha, a2, r, m, F0[3];
    const double* kd;
} adj_pixel;

static int adj_setup(const double* P, const double* cam, adj_pixel* A) {
    double N[3] = {P[0], P[1], P[2]};
    A->lN = norm3(N);
    if (!(A->lN > 0.0)) return 0;
    for (int k = 0; k < 3; ++k) A->n[k] = N[k] / A->lN;
    A->kd = P + 3;
    A->r = P[7];
    A->m = P[8];
    A->alpha = orc_alpha(A->r);
    A->a2 = A->alpha * A->alpha;
    sub3(cam, P + 9, A->wo);
    normalize3(A->wo);
    A->co = dot3(A->n, A->wo);
    for (int c = 0; c < 3; ++c) A->F0[c] = 0.04 * (1.0 - A->m) + A->kd[c] * A->m;
    return 1;
}

/* Contribution of one frozen sample to the gradient: dL/dn (unprojected,
 * including the view-cosine term along wo), dL/dalpha, dL/dF0 and dL/dtexel.
 * With mag != NULL it also returns the same quantities evaluated with every
 * sum replaced by the sum of its terms' absolute values (upstream gradients
 * may have either sign): mag->dn_terms holds the four vector terms of dL/dn
 * separately (cosine of the diffuse part, cosine of the specular part, half
 * vector, view), so that the caller can bound them after projection. */
static double dd_safe(double nh, double a2) { return nh * nh * (a2 - 1.0) + 1.0; }

typedef struct {
    double dn_terms[4][3];
    double dalpha, dF0[3], dL[3];
} adj_mag;

static void adj_sample(const adj_pixel* A, const orc_sample_rec* s, int spec_on, const double* L, const double* gd,
                       const double* gs, double dn[3], double* dalpha, double dF0[3], double dL[3], adj_mag* mag) {
    const double* n = A->n;
    const double* wo = A->wo;
    double a = s->vis * s->inv_denom;
    double ci = dot3(n, s->wi);
    double g_ci = 0.0, g_co = 0.0, g_nh = 0.0, h[3] = {0, 0, 0};
    double m_ci_d = 0.0, m_ci_s = 0.0, m_co = 0.0, m_nh = 0.0;
    *dalpha = 0.0;
    if (mag) memset(mag, 0, sizeof(*mag));
    /* diffuse: c_d,c = a L_c ci / pi */
    for (int c = 0; c < 3; ++c) {
        dL[c] = a * gd[c] * ci / ORC_PI;
        dF0[c] = 0.0;
        g_ci += a * gd[c] * L[c] / ORC_PI;
        if (mag) {
            mag->dL[c] = fabs(dL[c]);
            m_ci_d += fabs(a * gd[c] * L[c] / ORC_PI);
        }
    }
    if (spec_on) {
        double alpha = A->alpha, a2 = A->a2, co = A->co;
        for (int k = 0; k < 3; ++k) h[k] = s->wi[k] + wo[k];
        normalize3(h);
        double nh = dot3(n, h), vh = dot3(wo, h);
        double D = orc_ggx_D(nh, alpha);
        double li = orc_ggx_lambda(ci, alpha), lo = orc_ggx_lambda(co, alpha);
        double G2 = 1.0 / (1.0 + li + lo);
        double S = D * G2 / (4.0 * co); /* c_s,c = a L_c S F_c */
        double x = 1.0 - (vh < 0.0 ? 0.0 : (vh > 1.0 ? 1.0 : vh));
        double q5 = x * x * x * x * x;
        double gS = 0.0, mS = 0.0;
        for (int c = 0; c < 3; ++c) {
            double F = A->F0[c] + (1.0 - A->F0[c]) * q5;
            dL[c] += a * gs[c] * S * F;
            gS += a * gs[c] * L[c] * F;
            dF0[c] = a * gs[c] * L[c] * S * (1.0 - q5);
            if (mag) {
                mag->dL[c] += fabs(a * gs[c] * S * F);
                mS += fabs(a * gs[c] * L[c] * F);
                mag->dF0[c] = fabs(dF0[c]);
            }
        }
        /* S = D(nh, alpha) G2(Lambda_i, Lambda_o) / (4 co) */
        double dD_dnh = 0.0, dD_dalpha = 0.0;
        if (nh > 0.0) {
            double dd = nh * nh * (a2 - 1.0) + 1.0;
            dD_dnh = -4.0 * D * nh * (a2 - 1.0) / dd;
            dD_dalpha = D * (2.0 / alpha - 4.0 * alpha * nh * nh / dd);
        }
        /* Lambda(c) = (sqrt(1+z)-1)/2, z = alpha^2 (1/c^2 - 1) */
        double zi = a2 * (1.0 / (ci * ci) - 1.0), zo = a2 * (1.0 / (co * co) - 1.0);
        double si = sqrt(1.0 + zi), so = sqrt(1.0 + zo);
        double dli_dci = (1.0 / (4.0 * si)) * (-2.0 * a2 / (ci * ci * ci));
        double dlo_dco = (1.0 / (4.0 * so)) * (-2.0 * a2 / (co * co * co));
        double dli_dalpha = (1.0 / (4.0 * si)) * 2.0 * alpha * (1.0 / (ci * ci) - 1.0);
        double dlo_dalpha = (1.0 / (4.0 * so)) * 2.0 * alpha * (1.0 / (co * co) - 1.0);
        double dS_dD = G2 / (4.0 * co);
        double dS_dLam = -D * G2 * G2 / (4.0 * co); /* dG2/dLambda = -G2^2 */
        g_nh = gS * dS_dD * dD_dnh;
        *dalpha = gS * (dS_dD * dD_dalpha + dS_dLam * (dli_dalpha + dlo_dalpha));
        g_ci += gS * dS_dLam * dli_dci;
        g_co = gS * (dS_dLam * dlo_dco - S / co);
        if (mag) {
            m_nh = fabs(mS * dS_dD * dD_dnh);
            mag->dalpha = mS * (fabs(dS_dD * D * 2.0 / alpha) + fabs(dS_dD * D * 4.0 * alpha * nh * nh / dd_safe(nh, a2)) +
                                fabs(dS_dLam * dli_dalpha) + fabs(dS_dLam * dlo_dalpha));
            m_ci_s = fabs(mS * dS_dLam * dli_dci);
            m_co = mS * (fabs(dS_dLam * dlo_dco) + fabs(S / co));
        }
    }
    for (int k = 0; k < 3; ++k) dn[k] = g_ci * s->wi[k] + g_nh * h[k] + g_co * wo[k];
    if (mag) {
        for (int k = 0; k < 3; ++k) {
            mag->dn_terms[0][k] = m_ci_d * s->wi[k];
            mag->dn_terms[1][k] = m_ci_s * s->wi[k];
            mag->dn_terms[2][k] = m_nh * h[k];
            mag->dn_terms[3][k] = m_co * wo[k];
        }
    }
}

/* n = N / |N|:  dL/dN = (I - n n^T) dL/dn / |N| */
static void adj_project(const adj_pixel* A, const double gn[3], double out[3]) {
    double ng = dot3(A->n, gn);
    for (int k = 0; k < 3; ++k) out[k] = (gn[k] - A->n[k] * ng) / A->lN;
}

/* Analytic adjoint of orc_frozen_eval for the scalar  sum_q <g_q, out_q>.
 * g: 9 per pixel (dL/dc_d, dL/dk_d,out, dL/dc_s).
 * Writes grad: 9 per pixel (dL/dN.xyz, dL/dk_d.rgb, dL/d(o,r,m)) and
 * accumulates dL/dtexel into genv3 (3 per texel; serial over pixels).
 * With scale != NULL it also writes, per pixel and component, the sum of the
 * absolute values of the per-sample contributions (and accumulates the same
 * for the texels into genv3_scale): the magnitude a floating-point summation
 * error of the gradient is measured against. */
void orc_frozen_adjoint(const orc_sample_rec* recs, int spp, int n_pix, const double* prow, const double* cam_pos,
                        const int* spec_on, const double* env3, const double* g, double* grad, double* genv3,
                        double* scale, double* genv3_scale) {
    for (int q = 0; q < n_pix; ++q) {
        const double* gd = g + 9 * (size_t)q;
        const double* gk = gd + 3;
        const double* gs = gd + 6;
        double* G = grad + 9 * (size_t)q;
        double* Sc = scale ? scale + 9 * (size_t)q : NULL;
        memset(G, 0, 9 * sizeof(double));
        if (Sc) memset(Sc, 0, 9 * sizeof(double));
        adj_pixel A;
        if (!adj_setup(prow + 12 * (size_t)q, cam_pos + 3 * (size_t)q, &A)) continue;
        double gn[3] = {0, 0, 0}, g_alpha = 0.0, gF0[3] = {0, 0, 0};
        const double* kd = A.kd;
        double m = A.m, r = A.r;
        int r_live = r * r > 1e-4;
        for (int j = 0; j < spp; ++j) {
            const orc_sample_rec* s = recs + (size_t)q * spp + j;
            if (!s->active) continue;
            double dn[3], da, dF0[3], dL[3];
            adj_mag M;
            adj_sample(&A, s, spec_on[q], env3 + 3 * (size_t)s->texel, gd, gs, dn, &da, dF0, dL, Sc ? &M : NULL);
            double* gL = genv3 + 3 * (size_t)s->texel;
            for (int k = 0; k < 3; ++k) {
                gn[k] += dn[k];
                gF0[k] += dF0[k];
                gL[k] += dL[k];
            }
            g_alpha += da;
            if (Sc) {
                for (int t = 0; t < 4; ++t) {
                    double pn[3];
                    adj_project(&A, M.dn_terms[t], pn);
                    for (int k = 0; k < 3; ++k) Sc[k] += fabs(pn[k]);
                }
                for (int k = 0; k < 3; ++k) {
                    Sc[3 + k] += M.dF0[k] * fabs(m);
                    Sc[8] += M.dF0[k] * fabs(kd[k] - 0.04);
                    genv3_scale[3 * (size_t)s->texel + k] += M.dL[k];
                }
                Sc[7] += r_live ? M.dalpha * 2.0 * fabs(r) : 0.0;
            }
        }
        adj_project(&A, gn, G);
        double g_m = 0.0, dmk = 0.0;
        for (int c = 0; c < 3; ++c) {
            G[3 + c] = gk[c] * (1.0 - m) + gF0[c] * m;
            g_m += -gk[c] * kd[c] + gF0[c] * (kd[c] - 0.04);
            dmk += fabs(gk[c] * kd[c]);
            if (Sc) Sc[3 + c] += fabs(gk[c] * (1.0 - m));
        }
        if (Sc) Sc[8] += dmk;
        G[6] = 0.0;
        G[7] = r_live ? g_alpha * 2.0 * r : 0.0;
        G[8] = g_m;
    }
}

/* size of the record struct, so the Python side can check its mirror */
int orc_sample_rec_size(void) { return (int)sizeof(orc_sample_rec); }

/* ------------------------------------------------------------------------ */
/* Batch forms of the scalar functions above, for the quadrature and         */
/* histogram checks of the test suite (loops over the scalar functions).    */
/* ------------------------------------------------------------------------ */
void orc_pdf_light_n(const float* cond32, const float* marg32, int W, int H, double total, const double* dirs,
                     int n, double* out) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < n; ++k) out[k] = orc_pdf_light(cond32, marg32, W, H, total, dirs + 3 * (size_t)k);
}

void orc_sample_light_n(const float* cond32, const float* marg32, int W, int H, double total, const double* u,
                        int n, double* dirs, int* texels, double* pdfs) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < n; ++k) {
        if (!orc_sample_light(cond32, marg32, W, H, total, u[2 * k], u[2 * k + 1], dirs + 3 * (size_t)k,
                              texels + k, pdfs + k, NULL)) {
            texels[k] = -1;
            pdfs[k] = 0.0;
        }
    }
}

void orc_sample_cosine_n(const double nrm[3], const double* u, int n, double* dirs) {
    for (int k = 0; k < n; ++k) orc_sample_cosine(nrm, u[2 * k], u[2 * k + 1], dirs + 3 * (size_t)k);
}

void orc_pdf_cosine_n(const double nrm[3], const double* dirs, int n, double* out) {
    for (int k = 0; k < n; ++k) out[k] = orc_pdf_cosine(nrm, dirs + 3 * (size_t)k);
}

void orc_sample_ggx_n(const double nrm[3], const double wo[3], double alpha, const double* u, int n, double* dirs) {
    for (int k = 0; k < n; ++k) orc_sample_ggx(nrm, wo, alpha, u[2 * k], u[2 * k + 1], dirs + 3 * (size_t)k);
}

void orc_pdf_ggx_n(const double nrm[3], const double wo[3], double alpha, const double* dirs, int n, double* out) {
    for (int k = 0; k < n; ++k) out[k] = orc_pdf_ggx(nrm, wo, alpha, dirs + 3 * (size_t)k);
}

void orc_ggx_D_n(const double* nh, int n, double alpha, double* out) {
    for (int k = 0; k < n; ++k) out[k] = orc_ggx_D(nh[k], alpha);
}

void orc_ggx_G2_n(const double* ci, const double* co, int n, double alpha, double* out) {
    for (int k = 0; k < n; ++k) out[k] = orc_ggx_G2(ci[k], co[k], alpha);
}

/* ------------------------------------------------------------------------ */
/* 10. Shadow-visibility gradients by edge sampling (App. "Visibility        */
/*     gradients from shadows"; Sec. 3.1 "Shadow gradients").  The paper      */
/*     evaluates these gradients as an ablation, citing reparameterisation    */
/*     (Loubet et al. 2019) and warped-area sampling (Bangaru et al. 2020),   */
/*     and leaves them off by default.  Reading taken here: the boundary term */
/*     of the direct-illumination integral, estimated by edge sampling in the */
/*     manner of Li et al. 2018, for the vertex positions of the occluders.   */
/*                                                                            */
/*     With H = 1 - tau B (B the blocked indicator of the shadow ray from     */
/*     o = p + eps n), the pixel's integral I = int g(w) (1 - tau B(w)) dw    */
/*     moves with the mesh only through the boundary of the blocked set:      */
/*       dI = -tau sum_silhouette-edges int_0^1 g(w(s)) V+(s) (n_out . dx(s)) */
/*                                   |w x (b - a)| / r^2 ds,                  */
/*     x(s) = a + s (b - a), r = |x - o|, w = (x - o)/r, dx = (1-s) da + s db */
/*     n_out the unit normal of the plane (o, a, b) on the side away from the */
/*     edge's faces, and V+ = 1 when the ray leaving o just outside the edge  */
/*     (along w + eta n_out, normalised) reaches the probe.  g(w) is the      */
/*     integrand of the forward estimator weighted by the upstream gradient: */
/*       g = sum_c L_c(w) [ gcd_c (n.w)/pi + gcs_c D G2 F_c / (4 n.wo) ],      */
/*     with (n.w) > 0 required and the specular term only where the lobe is  */
/*     on.  An edge is on the silhouette seen from o when its two faces lie   */
/*     on the same side of the plane (o, a, b) (strictly), or when it has one */
/*     face.  Estimator: per pixel M samples, each an edge drawn uniformly    */
/*     (e = floor(u0 E) from the 24-bit uniform, computed exactly in integer  */
/*     arithmetic) and s = u1 uniform, weighted by E / M.                      */
/* ------------------------------------------------------------------------ */

/* Edge table: one record (a, b, c1, c2) per undirected edge, in the order of
 * the edge's first half-edge h = 3 t + i (a = v_i, b = v_(i+1), c1 = v_(i+2)
 * of that triangle); c2 is the opposite vertex of the next half-edge with the
 * same endpoints (-1 for a boundary edge; further faces of a non-manifold
 * edge are ignored).  Returns the number of edges. */
typedef struct {
    uint64_t key;
    int h;
} orc_half_edge;

static int cmp_half_edge(const void* x, const void* y) {
    const orc_half_edge* a = (const orc_half_edge*)x;
    const orc_half_edge* b = (const orc_half_edge*)y;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->h < b->h ? -1 : (a->h > b->h);
}

int orc_edge_table(const int* tris, int n_tris, int* edges) {
    const int nh = 3 * n_tris;
    orc_half_edge* he = (orc_half_edge*)malloc(sizeof(orc_half_edge) * (size_t)(nh > 0 ? nh : 1));
    int* second = (int*)malloc(sizeof(int) * (size_t)(nh > 0 ? nh : 1)); /* owner h -> next half-edge or -1 */
    int* owner = (int*)malloc(sizeof(int) * (size_t)(nh > 0 ? nh : 1));
    for (int h = 0; h < nh; ++h) {
        int t = h / 3, i = h % 3;
        uint32_t a = (uint32_t)tris[3 * t + i], b = (uint32_t)tris[3 * t + (i + 1) % 3];
        uint32_t lo = a < b ? a : b, hi = a < b ? b : a;
        he[h].key = ((uint64_t)lo << 32) | hi;
        he[h].h = h;
        owner[h] = 0;
        second[h] = -1;
    }
    qsort(he, (size_t)nh, sizeof(orc_half_edge), cmp_half_edge);
    for (int k = 0; k < nh;) {
        int l = k;
        while (l < nh && he[l].key == he[k].key) ++l;
        owner[he[k].h] = 1;
        if (l - k > 1) second[he[k].h] = he[k + 1].h;
        k = l;
    }
    int n = 0;
    for (int h = 0; h < nh; ++h) {
        if (!owner[h]) continue;
        int t = h / 3, i = h % 3;
        edges[4 * n] = tris[3 * t + i];
        edges[4 * n + 1] = tris[3 * t + (i + 1) % 3];
        edges[4 * n + 2] = tris[3 * t + (i + 2) % 3];
        if (second[h] >= 0) {
            int t2 = second[h] / 3, i2 = second[h] % 3;
            edges[4 * n + 3] = tris[3 * t2 + (i2 + 2) % 3];
        } else {
            edges[4 * n + 3] = -1;
        }
        ++n;
    }
    free(he);
    free(second);
    free(owner);
    return n;
}

typedef struct {
    uint64_t seed;
    uint32_t stream;
    int n_samples; /* M, edge samples per pixel */
    double tau, ray_eps, eta;
} orc_edge_params;

/* gb, cam_pos, ctr as in orc_shade_fwd; gcd, gcs: 3 doubles per pixel (the
 * upstream gradients of c_d and c_s).  g_verts (3 per vertex) is accumulated.
 * rec (nullable): 4 doubles per sample: the signed weight -tau g J E / M of a
 * contributing sample (0 otherwise), the distance to the nearest discrete
 * decision (silhouette side, horizon, outer ray, probe texel), the edge index
 * and s. */
void orc_shadow_edge_grad(const float* verts, const int* tris, int n_tris, const int* edges, int n_edges,
                          const float* env, int W, int H, const float* gb, const double* cam_pos, const uint32_t* ctr,
                          int n_pix, const double* gcd, const double* gcs, orc_edge_params prm, double* g_verts,
                          double* rec) {
    const int M = prm.n_samples;
    for (int q = 0; q < n_pix; ++q) {
        const float* g = gb + 16 * (size_t)q;
        double* rq = rec ? rec + 4 * (size_t)q * M : NULL;
        if (rq) memset(rq, 0, 4 * (size_t)M * sizeof(double));
        double N[3] = {g[4], g[5], g[6]};
        double lN = norm3(N);
        if (!(g[3] > 0.0) || !(lN > 0.0) || n_edges <= 0) continue;
        double n[3] = {N[0] / lN, N[1] / lN, N[2] / lN};
        double o[3] = {g[0] + prm.ray_eps * n[0], g[1] + prm.ray_eps * n[1], g[2] + prm.ray_eps * n[2]};
        double kd[3] = {g[8], g[9], g[10]};
        double m_ = g[14], alpha = orc_alpha(g[13]);
        double p[3] = {g[0], g[1], g[2]}, wo[3];
        sub3(cam_pos + 3 * (size_t)q, p, wo);
        normalize3(wo);
        double co = dot3(n, wo);
        int spec_on = co >= 1e-4;
        const double* gd = gcd + 3 * (size_t)q;
        const double* gs = gcs + 3 * (size_t)q;
        for (int j = 0; j < M; ++j) {
            double u[2];
            orc_sample_uniforms(prm.seed, ctr[2 * q], ctr[2 * q + 1], (uint32_t)j, prm.stream, u);
            /* u0 = k 2^-24 exactly, so u0 * E is exact in double and floor is the integer rule */
            int e = (int)floor(u[0] * (double)n_edges);
            double s = u[1];
            double* r = rq ? rq + 4 * (size_t)j : NULL;
            if (r) {
                r[1] = INFINITY;
                r[2] = e;
                r[3] = s;
            }
            const int* E4 = edges + 4 * (size_t)e;
            double va[3], vb[3], vc[3], A[3], B[3], mm[3], t3[3];
            load_vert(verts, E4[0], va);
            load_vert(verts, E4[1], vb);
            sub3(va, o, A);
            sub3(vb, o, B);
            cross3(A, B, mm);
            double lm = norm3(mm);
            if (!(lm > 0.0)) continue;
            load_vert(verts, E4[2], vc);
            sub3(vc, o, t3);
            double s1 = dot3(mm, t3) / (lm * norm3(t3));
            double s2 = s1;
            if (E4[3] >= 0) {
                load_vert(verts, E4[3], vc);
                sub3(vc, o, t3);
                s2 = dot3(mm, t3) / (lm * norm3(t3));
            }
            double margin = fabs(s1) < fabs(s2) ? fabs(s1) : fabs(s2);
            if (r) r[1] = margin;
            if (!(s1 * s2 > 0.0)) continue; /* not on the silhouette seen from o */
            double x[3], d[3], w[3], ab[3];
            sub3(vb, va, ab);
            for (int c = 0; c < 3; ++c) x[c] = va[c] + s * ab[c];
            sub3(x, o, d);
            double rr = norm3(d);
            for (int c = 0; c < 3; ++c) w[c] = d[c] / rr;
            double ci = dot3(n, w);
            if (fabs(ci) < margin) margin = fabs(ci);
            if (r) r[1] = margin;
            if (!(ci > 0.0)) continue;
            double sg = s1 > 0.0 ? -1.0 : 1.0, nout[3], wp[3];
            for (int c = 0; c < 3; ++c) {
                nout[c] = sg * mm[c] / lm;
                wp[c] = w[c] + prm.eta * nout[c];
            }
            normalize3(wp);
            double em, tm;
            int blocked = orc_any_hit(verts, tris, n_tris, o, wp, &em, &tm);
            if (em < margin) margin = em;
            if (tm < margin) margin = tm;
            double bd;
            int texel = orc_texel_of_dir(w, W, H, &bd);
            if (bd < margin) margin = bd;
            if (r) r[1] = margin;
            if (blocked) continue;
            const float* L = env + 4 * (size_t)texel;
            double gw = 0.0;
            for (int c = 0; c < 3; ++c) gw += L[c] * gd[c] * ci / ORC_PI;
            if (spec_on) {
                double h[3] = {w[0] + wo[0], w[1] + wo[1], w[2] + wo[2]};
                normalize3(h);
                double D = orc_ggx_D(dot3(n, h), alpha);
                double G2 = orc_ggx_G2(ci, co, alpha);
                double vh = dot3(wo, h);
                for (int c = 0; c < 3; ++c) {
                    double F0 = 0.04 * (1.0 - m_) + kd[c] * m_;
                    gw += L[c] * gs[c] * D * G2 * orc_schlick(F0, vh) / (4.0 * co);
                }
            }
            double wxab[3];
            cross3(w, ab, wxab);
            double J = norm3(wxab) / (rr * rr);
            double wt = -prm.tau * gw * J * (double)n_edges / (double)M;
            if (r) r[0] = wt;
            for (int c = 0; c < 3; ++c) {
                g_verts[3 * (size_t)E4[0] + c] += wt * (1.0 - s) * nout[c];
                g_verts[3 * (size_t)E4[1] + c] += wt * s * nout[c];
            }
        }
    }
}
