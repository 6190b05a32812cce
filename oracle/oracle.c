/*
 * Plain, slow CPU oracle for the EngineCL hot path (Nozal, Bosque, Beivide,
 * "EngineCL: Usability and Performance in Heterogeneous Computing").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or constant
 * with the CUDA path: the two meet only through the seeded input arrays.
 *
 * Every routine is the plain definition of what one work-group range of a
 * kernel computes, evaluated in double precision unless the method itself
 * fixes the precision (the Mandelbrot escape count is an FP32 computation
 * whose integer result is compared bit for bit).  Each routine takes a
 * half-open range of independent units [begin, end) so that the Python
 * wrapper can spread large cases over host threads; there is no blocking,
 * fusion or reordering beyond that.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC (the
 * contraction switch matters: a fused multiply-add in the Mandelbrot loop
 * would change iteration counts).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Mandelbrot (Sec. 5.3 Fig. 6 workload; Table 2: lws 256, 0:1 buffers,
 * out pattern 4:1).  Pixel (i, j) maps to c = (x0 + i*dx, y0 + j*dy).
 * z starts at 0; while fewer than max_iter steps were taken and
 * |z|^2 <= 4, z <- z^2 + c and the count grows by one.  The count is the
 * output.  Every operation is one correctly rounded FP32 operation in the
 * order written, no fused multiply-add.
 */
void ecl_oracle_mandelbrot(uint32_t *out, int64_t width, int64_t height,
                           float x0, float y0, float dx, float dy,
                           int32_t max_iter, int64_t row_begin, int64_t row_end)
{
    (void)height;
    for (int64_t j = row_begin; j < row_end; ++j) {
        for (int64_t i = 0; i < width; ++i) {
            float cx = x0 + (float)i * dx;
            float cy = y0 + (float)j * dy;
            float x = 0.0f, y = 0.0f;
            int32_t n = 0;
            while (n < max_iter) {
                float x2 = x * x;
                float y2 = y * y;
                if (x2 + y2 > 4.0f) break;
                float xt = (x2 - y2) + cx;
                y = (2.0f * x) * y + cy;
                x = xt;
                ++n;
            }
            out[j * width + i] = (uint32_t)n;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Gaussian blur (Table 2: lws 128, image + filter-weight buffers, out
 * pattern 1:1).  Separable filter with clamp-to-edge borders:
 *   out[y][x] = sum_v w[v] * sum_u w[u] * in[clamp(y+v-r)][clamp(x+u-r)]
 * with r = taps/2, evaluated as a horizontal pass followed by a vertical
 * pass, both in double precision.  Rows [row_begin, row_end) are produced.
 */
static int64_t clampi(int64_t v, int64_t lo, int64_t hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

void ecl_oracle_gaussian(const float *in, int64_t width, int64_t height,
                         const float *w, int32_t taps, double *out,
                         int64_t row_begin, int64_t row_end)
{
    const int64_t r = taps / 2;
    const int64_t nrows = (row_end - row_begin) + 2 * r;
    double *h = (double *)malloc(sizeof(double) * (size_t)(nrows * width));
    if (!h) return;
    /* horizontal pass over the rows the vertical pass needs */
    for (int64_t t = 0; t < nrows; ++t) {
        const int64_t ys = clampi(row_begin - r + t, 0, height - 1);
        for (int64_t x = 0; x < width; ++x) {
            double s = 0.0;
            for (int64_t u = 0; u < taps; ++u)
                s += (double)w[u] * (double)in[ys * width + clampi(x + u - r, 0, width - 1)];
            h[t * width + x] = s;
        }
    }
    /* vertical pass */
    for (int64_t y = row_begin; y < row_end; ++y) {
        const int64_t t0 = y - row_begin;
        for (int64_t x = 0; x < width; ++x) {
            double s = 0.0;
            for (int64_t v = 0; v < taps; ++v)
                s += (double)w[v] * h[(t0 + v) * width + x];
            out[y * width + x] = s;
        }
    }
    free(h);
}

/* Direct two-dimensional sum of the same filter (taps*taps terms per
 * pixel).  Used only to pin the separable evaluation on small images. */
void ecl_oracle_gaussian_direct(const float *in, int64_t width, int64_t height,
                                const float *w, int32_t taps, double *out)
{
    const int64_t r = taps / 2;
    for (int64_t y = 0; y < height; ++y)
        for (int64_t x = 0; x < width; ++x) {
            double s = 0.0;
            for (int64_t v = 0; v < taps; ++v)
                for (int64_t u = 0; u < taps; ++u)
                    s += (double)w[v] * (double)w[u] *
                         (double)in[clampi(y + v - r, 0, height - 1) * width +
                                    clampi(x + u - r, 0, width - 1)];
            out[y * width + x] = s;
        }
}

/* ------------------------------------------------------------------ */
/* NBody (Listing 2: float4 positions, softening passed squared).
 * pos4[4*i] = (x, y, z, m).  Gravitational constant 1.
 *   a_i = sum_j m_j (r_j - r_i) / (|r_j - r_i|^2 + eps2)^(3/2)
 * The sum runs over every j, the self term included (it is exactly 0).
 */
static void acc_one(const float *pos4, int64_t n, double eps2, int64_t i, double *a)
{
    const double xi = pos4[4 * i], yi = pos4[4 * i + 1], zi = pos4[4 * i + 2];
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        const double dx = (double)pos4[4 * j] - xi;
        const double dy = (double)pos4[4 * j + 1] - yi;
        const double dz = (double)pos4[4 * j + 2] - zi;
        const double r2 = dx * dx + dy * dy + dz * dz + eps2;
        const double s = (double)pos4[4 * j + 3] / (r2 * sqrt(r2));
        ax += s * dx;
        ay += s * dy;
        az += s * dz;
    }
    a[0] = ax;
    a[1] = ay;
    a[2] = az;
}

void ecl_oracle_nbody_acc(const float *pos4, int64_t n, double eps2,
                          double *acc3, int64_t i_begin, int64_t i_end)
{
    for (int64_t i = i_begin; i < i_end; ++i) acc_one(pos4, n, eps2, i, acc3 + 3 * i);
}

/* One explicit step of the Listing 2 kernel shape (in pos/vel -> out
 * pos/vel): r' = r + v dt + a dt^2 / 2, v' = v + a dt, mass carried over. */
void ecl_oracle_nbody_step(const float *pos4, const float *vel4, int64_t n,
                           double dt, double eps2, double *pos_out4,
                           double *vel_out4, int64_t i_begin, int64_t i_end)
{
    double a[3];
    for (int64_t i = i_begin; i < i_end; ++i) {
        acc_one(pos4, n, eps2, i, a);
        for (int c = 0; c < 3; ++c) {
            pos_out4[4 * i + c] = (double)pos4[4 * i + c] + (double)vel4[4 * i + c] * dt +
                                  0.5 * a[c] * dt * dt;
            vel_out4[4 * i + c] = (double)vel4[4 * i + c] + a[c] * dt;
        }
        pos_out4[4 * i + 3] = pos4[4 * i + 3];
        vel_out4[4 * i + 3] = vel4[4 * i + 3];
    }
}

/* Potential energy E = - sum_{i<j} m_i m_j / sqrt(|r_i - r_j|^2 + eps2).
 * Returns the part of the sum whose first index lies in [i_begin, i_end). */
double ecl_oracle_nbody_energy(const float *pos4, int64_t n, double eps2,
                               int64_t i_begin, int64_t i_end)
{
    double e = 0.0;
    for (int64_t i = i_begin; i < i_end; ++i) {
        const double xi = pos4[4 * i], yi = pos4[4 * i + 1], zi = pos4[4 * i + 2];
        const double mi = pos4[4 * i + 3];
        double row = 0.0;
        for (int64_t j = i + 1; j < n; ++j) {
            const double dx = xi - (double)pos4[4 * j];
            const double dy = yi - (double)pos4[4 * j + 1];
            const double dz = zi - (double)pos4[4 * j + 2];
            row += (double)pos4[4 * j + 3] / sqrt(dx * dx + dy * dy + dz * dz + eps2);
        }
        e -= mi * row;
    }
    return e;
}

/* The terms of E that involve body i, with body i placed at q[0..2]:
 *   - m_i * sum_{j != i} m_j / sqrt(|q - r_j|^2 + eps2).
 * E(q) - E(q') equals the difference of this row for two placements of
 * body i, which is what a finite difference in one coordinate needs. */
double ecl_oracle_nbody_energy_row(const float *pos4, int64_t n, double eps2,
                                   int64_t i, const double *q)
{
    double row = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        const double dx = q[0] - (double)pos4[4 * j];
        const double dy = q[1] - (double)pos4[4 * j + 1];
        const double dz = q[2] - (double)pos4[4 * j + 2];
        row += (double)pos4[4 * j + 3] / sqrt(dx * dx + dy * dy + dz * dz + eps2);
    }
    return -(double)pos4[4 * i + 3] * row;
}

/* Gradient of E with respect to r_i, differentiated term by term:
 *   dE/dr_i = sum_{j != i} m_i m_j (r_i - r_j) / (|r_i - r_j|^2 + eps2)^(3/2) */
void ecl_oracle_nbody_energy_grad(const float *pos4, int64_t n, double eps2,
                                  double *grad3, int64_t i_begin, int64_t i_end)
{
    for (int64_t i = i_begin; i < i_end; ++i) {
        const double xi = pos4[4 * i], yi = pos4[4 * i + 1], zi = pos4[4 * i + 2];
        const double mi = pos4[4 * i + 3];
        double gx = 0.0, gy = 0.0, gz = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            const double dx = xi - (double)pos4[4 * j];
            const double dy = yi - (double)pos4[4 * j + 1];
            const double dz = zi - (double)pos4[4 * j + 2];
            const double r2 = dx * dx + dy * dy + dz * dz + eps2;
            const double s = mi * (double)pos4[4 * j + 3] / (r2 * sqrt(r2));
            gx += s * dx;
            gy += s * dy;
            gz += s * dz;
        }
        grad3[3 * i] = gx;
        grad3[3 * i + 1] = gy;
        grad3[3 * i + 2] = gz;
    }
}

/* Potential of body i: phi_i = sum_{j != i} m_j / sqrt(|r_i - r_j|^2 + eps2),
 * so that dE/dm_i = -phi_i and sum_i m_i phi_i = -2E. */
void ecl_oracle_nbody_potential(const float *pos4, int64_t n, double eps2, double *phi,
                                int64_t i_begin, int64_t i_end)
{
    for (int64_t i = i_begin; i < i_end; ++i) {
        const double xi = pos4[4 * i], yi = pos4[4 * i + 1], zi = pos4[4 * i + 2];
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            const double dx = xi - (double)pos4[4 * j];
            const double dy = yi - (double)pos4[4 * j + 1];
            const double dz = zi - (double)pos4[4 * j + 2];
            s += (double)pos4[4 * j + 3] / sqrt(dx * dx + dy * dy + dz * dz + eps2);
        }
        phi[i] = s;
    }
}

/* ------------------------------------------------------------------ */
/* Binomial options (Listing 1 workload): Cox-Ross-Rubinstein lattice for a
 * European option, priced by backward induction, with the exact
 * derivatives of the discrete price with respect to spot S and volatility
 * sigma carried along in forward mode (dual numbers).
 *   dt = T/N, u = exp(sigma sqrt(dt)), d = 1/u,
 *   p = (exp(r dt) - d) / (u - d), disc = exp(-r dt)
 *   leaf j (j up-moves): S u^j d^(N-j), payoff max(S_T - K, 0) for a call,
 *   max(K - S_T, 0) for a put
 *   V_j <- disc * (p V_{j+1} + (1 - p) V_j), N times.
 */
typedef struct { double v, ds, dv; } dual3; /* value, d/dS, d/dsigma */

static dual3 d3(double v, double ds, double dv) { dual3 r = {v, ds, dv}; return r; }
static dual3 d3add(dual3 a, dual3 b) { return d3(a.v + b.v, a.ds + b.ds, a.dv + b.dv); }
static dual3 d3sub(dual3 a, dual3 b) { return d3(a.v - b.v, a.ds - b.ds, a.dv - b.dv); }
static dual3 d3mul(dual3 a, dual3 b)
{
    return d3(a.v * b.v, a.ds * b.v + a.v * b.ds, a.dv * b.v + a.v * b.dv);
}
static dual3 d3div(dual3 a, dual3 b)
{
    const double q = a.v / b.v;
    return d3(q, (a.ds - q * b.ds) / b.v, (a.dv - q * b.dv) / b.v);
}
static dual3 d3exp(dual3 a)
{
    const double e = exp(a.v);
    return d3(e, e * a.ds, e * a.dv);
}

void ecl_oracle_binomial(const float *S, const float *K, const float *T,
                         const float *sigma, const int32_t *steps, double r,
                         int32_t put, int64_t begin, int64_t end,
                         double *price, double *delta, double *vega)
{
    int32_t cap = 0;
    dual3 *V = NULL;
    for (int64_t o = begin; o < end; ++o) {
        const int32_t N = steps[o];
        if (N + 1 > cap) {
            free(V);
            cap = N + 1;
            V = (dual3 *)malloc(sizeof(dual3) * (size_t)cap);
            if (!V) return;
        }
        const double dt = (double)T[o] / (double)N;
        const dual3 Sd = d3(S[o], 1.0, 0.0);
        const dual3 sig = d3(sigma[o], 0.0, 1.0);
        const dual3 a = d3mul(sig, d3(sqrt(dt), 0.0, 0.0));
        const dual3 u = d3exp(a);
        const dual3 d = d3div(d3(1.0, 0.0, 0.0), u);
        const dual3 growth = d3(exp(r * dt), 0.0, 0.0);
        const dual3 p = d3div(d3sub(growth, d), d3sub(u, d));
        const dual3 q = d3sub(d3(1.0, 0.0, 0.0), p);
        const dual3 disc = d3(exp(-r * dt), 0.0, 0.0);
        const dual3 Kd = d3(K[o], 0.0, 0.0);
        for (int32_t j = 0; j <= N; ++j) {
            /* u^j d^(N-j) = exp((2j - N) a) */
            const dual3 g = d3exp(d3mul(a, d3((double)(2 * j - N), 0.0, 0.0)));
            const dual3 ST = d3mul(Sd, g);
            const dual3 pay = put ? d3sub(Kd, ST) : d3sub(ST, Kd);
            V[j] = pay.v > 0.0 ? pay : d3(0.0, 0.0, 0.0);
        }
        for (int32_t t = N - 1; t >= 0; --t)
            for (int32_t j = 0; j <= t; ++j)
                V[j] = d3mul(disc, d3add(d3mul(p, V[j + 1]), d3mul(q, V[j])));
        price[o] = V[0].v;
        if (delta) delta[o] = V[0].ds;
        if (vega) vega[o] = V[0].dv;
    }
    free(V);
}

/* ------------------------------------------------------------------ */
/* GEMM C = A B^T-stored: A is M x K row-major, Bt is N x K row-major (row j
 * of Bt is column j of B), C[i][j] = sum_k A[i][k] Bt[j][k].
 *
 * bfloat16 rounding from the IEEE 754 definition: keep the sign, the 8
 * exponent bits and the top 7 fraction bits of binary32, rounding the
 * dropped 16 bits to nearest, ties to even; NaN stays NaN.
 */
float ecl_oracle_bf16_round(float x)
{
    uint32_t b;
    memcpy(&b, &x, 4);
    if ((b & 0x7f800000u) == 0x7f800000u && (b & 0x007fffffu)) {
        b |= 0x00400000u; /* quiet NaN, kept a NaN after truncation */
        b &= 0xffff0000u;
    } else {
        const uint32_t low = b & 0xffffu;
        uint32_t hi = b >> 16;
        if (low > 0x8000u || (low == 0x8000u && (hi & 1u))) hi += 1u;
        b = hi << 16;
    }
    float y;
    memcpy(&y, &b, 4);
    return y;
}

void ecl_oracle_bf16_round_array(const float *in, float *out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) out[i] = ecl_oracle_bf16_round(in[i]);
}

/* Entries (ii[t], jj[t]) of the product, in double precision.
 *   mode 0: bf16(A) * bf16(B)        (the plain BF16 GEMM's exact value)
 *   mode 1: A * B in FP64 of the FP32 inputs (the compensated mode's target)
 *   mode 2: hi(A)hi(B) + hi(A)lo(B) + lo(A)hi(B) with hi = bf16(x),
 *           lo = bf16(x - hi) (FP32 subtraction): the three-product split's
 *           exact value.
 *   mode 3: the six-product split: x = h + m + l with h = bf16(x),
 *           m = bf16(x - h), l = bf16((x - h) - m) (FP32 subtractions), and
 *           C = hh + hm + mh + hl + lh + mm (the products of order up to
 *           2^-16 relative; ml, lm and ll are left out). */
void ecl_oracle_gemm_entries(const float *A, const float *Bt, int64_t M, int64_t N,
                             int64_t K, int32_t mode, const int64_t *ii,
                             const int64_t *jj, int64_t count, double *out)
{
    (void)M;
    (void)N;
    for (int64_t t = 0; t < count; ++t) {
        const float *a = A + ii[t] * K;
        const float *b = Bt + jj[t] * K;
        double s = 0.0;
        for (int64_t k = 0; k < K; ++k) {
            if (mode == 0) {
                s += (double)ecl_oracle_bf16_round(a[k]) * (double)ecl_oracle_bf16_round(b[k]);
            } else if (mode == 1) {
                s += (double)a[k] * (double)b[k];
            } else if (mode == 3) {
                const float ah = ecl_oracle_bf16_round(a[k]);
                const float ar = a[k] - ah;
                const float am = ecl_oracle_bf16_round(ar);
                const float al = ecl_oracle_bf16_round(ar - am);
                const float bh = ecl_oracle_bf16_round(b[k]);
                const float br = b[k] - bh;
                const float bm = ecl_oracle_bf16_round(br);
                const float bl = ecl_oracle_bf16_round(br - bm);
                s += (double)ah * (double)bh + (double)ah * (double)bm + (double)am * (double)bh +
                     (double)ah * (double)bl + (double)al * (double)bh + (double)am * (double)bm;
            } else {
                const float ah = ecl_oracle_bf16_round(a[k]);
                const float al = ecl_oracle_bf16_round(a[k] - ah);
                const float bh = ecl_oracle_bf16_round(b[k]);
                const float bl = ecl_oracle_bf16_round(b[k] - bh);
                s += (double)ah * (double)bh + (double)ah * (double)bl + (double)al * (double)bh;
            }
        }
        out[t] = s;
    }
}

/* ------------------------------------------------------------------ */
/* Ray tracing (Sec. 7 "Ray": an irregular ray tracer over a scene of
 * spheres and point lights; Table 2: lws 128, scene in / image out, 1:1).
 * The paper's ray tracer and scenes are not available, so the method here
 * is a plain Whitted tracer, evaluated in FP32 operation by operation (no
 * fused multiply-add) so that a GPU evaluation in the same order matches
 * bit for bit.
 *
 * Scene (floats): sphere k at s[12k..]: centre x y z, radius, colour r g b,
 * reflectivity, kd, ks, log2 of the specular exponent, pad; light l after
 * the spheres at L[8l..]: position x y z, pad, intensity r g b, pad.
 * Camera at the origin looking down -z: pixel (i, j) has direction
 * (u, v, -1) / |(u, v, -1)| with u = (2i + 1 - W) / H, v = (H - 2j - 1) / H.
 * A ray's nearest hit is the smallest t > eps over the spheres in index
 * order (the first of equal t wins).  At a hit p with normal
 * n = (p - c) / |p - c| (normalised, so a grazing hit that rounding puts off
 * the surface still shades with a unit normal):
 *   local = ka col + sum over lights not shadowed (a shadow ray from
 *   p + eps n towards the light hits a sphere before it) of
 *   kd (n.l) col I  [n.l > 0]  +  ks (r.(-d))^(2^e) I  [r.(-d) > 0],
 *   r = 2 (n.l) n - l.
 * Reflections are followed front to back: with weight w (1 at first),
 * colour += w (1 - refl) local and w *= refl while refl > 0 and the depth
 * is below max_depth (the ray continues from p + eps n along the unit
 * vector of d - 2 (d.n) n); otherwise colour += w local and the ray ends; a miss adds
 * w * background.  Output per pixel: r, g, b, and the number of rays traced
 * (camera, reflected and shadow rays) as a float. */
#define RAY_EPS 1e-3f

static int ray_nearest(const float *sph, int32_t ns, float ox, float oy, float oz, float dx, float dy,
                       float dz, float *t_out)
{
    int best = -1;
    float tb = 3.0e38f;
    for (int32_t k = 0; k < ns; ++k) {
        const float *s = sph + 12 * k;
        const float ocx = ox - s[0], ocy = oy - s[1], ocz = oz - s[2];
        const float b = ocx * dx + ocy * dy + ocz * dz;
        const float c = (ocx * ocx + ocy * ocy + ocz * ocz) - s[3] * s[3];
        const float disc = b * b - c;
        if (disc < 0.0f) continue;
        const float sq = sqrtf(disc);
        float t = -b - sq;
        if (!(t > RAY_EPS)) t = -b + sq;
        if (t > RAY_EPS && t < tb) {
            tb = t;
            best = (int)k;
        }
    }
    *t_out = tb;
    return best;
}

static int ray_blocked(const float *sph, int32_t ns, float ox, float oy, float oz, float dx, float dy, float dz,
                       float dist)
{
    for (int32_t k = 0; k < ns; ++k) {
        const float *s = sph + 12 * k;
        const float ocx = ox - s[0], ocy = oy - s[1], ocz = oz - s[2];
        const float b = ocx * dx + ocy * dy + ocz * dz;
        const float c = (ocx * ocx + ocy * ocy + ocz * ocz) - s[3] * s[3];
        const float disc = b * b - c;
        if (disc < 0.0f) continue;
        const float sq = sqrtf(disc);
        float t = -b - sq;
        if (!(t > RAY_EPS)) t = -b + sq;
        if (t > RAY_EPS && t < dist) return 1;
    }
    return 0;
}

void ecl_oracle_ray(const float *scene, int32_t ns, int32_t nl, int64_t width, int64_t height, float ka,
                    float bg_r, float bg_g, float bg_b, int32_t max_depth, float *out, int64_t row_begin,
                    int64_t row_end)
{
    const float *lights = scene + 12 * (int64_t)ns;
    const float inv = 1.0f / (float)height;
    for (int64_t j = row_begin; j < row_end; ++j) {
        for (int64_t i = 0; i < width; ++i) {
            const float u = (float)(2 * i + 1 - width) * inv;
            const float v = (float)(height - 2 * j - 1) * inv;
            const float len = sqrtf(u * u + v * v + 1.0f);
            float dx = u / len, dy = v / len, dz = -1.0f / len;
            float ox = 0.0f, oy = 0.0f, oz = 0.0f;
            float cr = 0.0f, cg = 0.0f, cb = 0.0f, w = 1.0f;
            int32_t rays = 1;
            for (int32_t depth = 0;; ++depth) {
                float t;
                const int k = ray_nearest(scene, ns, ox, oy, oz, dx, dy, dz, &t);
                if (k < 0) {
                    cr += w * bg_r;
                    cg += w * bg_g;
                    cb += w * bg_b;
                    break;
                }
                const float *s = scene + 12 * k;
                const float px = ox + t * dx, py = oy + t * dy, pz = oz + t * dz;
                const float qx = px - s[0], qy = py - s[1], qz = pz - s[2];
                const float ql = sqrtf(qx * qx + qy * qy + qz * qz);
                const float nx = qx / ql, ny = qy / ql, nz = qz / ql;
                const float sox = px + nx * RAY_EPS, soy = py + ny * RAY_EPS, soz = pz + nz * RAY_EPS;
                float lr = ka * s[4], lg = ka * s[5], lb = ka * s[6];
                const int32_t e = (int32_t)s[10];
                for (int32_t l = 0; l < nl; ++l) {
                    const float *L = lights + 8 * l;
                    float lx = L[0] - px, ly = L[1] - py, lz = L[2] - pz;
                    const float dist = sqrtf(lx * lx + ly * ly + lz * lz);
                    lx = lx / dist;
                    ly = ly / dist;
                    lz = lz / dist;
                    ++rays;
                    if (ray_blocked(scene, ns, sox, soy, soz, lx, ly, lz, dist)) continue;
                    const float ndl = nx * lx + ny * ly + nz * lz;
                    if (!(ndl > 0.0f)) continue;
                    const float dif = s[8] * ndl;
                    lr += (dif * s[4]) * L[4];
                    lg += (dif * s[5]) * L[5];
                    lb += (dif * s[6]) * L[6];
                    const float rx = (2.0f * ndl) * nx - lx, ry = (2.0f * ndl) * ny - ly,
                                rz = (2.0f * ndl) * nz - lz;
                    const float rdv = -(rx * dx + ry * dy + rz * dz);
                    if (rdv > 0.0f) {
                        float sp = rdv;
                        for (int32_t q = 0; q < e; ++q) sp = sp * sp;
                        const float spec = s[9] * sp;
                        lr += spec * L[4];
                        lg += spec * L[5];
                        lb += spec * L[6];
                    }
                }
                const float refl = s[7];
                if (refl > 0.0f && depth < max_depth) {
                    const float wl = w * (1.0f - refl);
                    cr += wl * lr;
                    cg += wl * lg;
                    cb += wl * lb;
                    w = w * refl;
                    const float dn = dx * nx + dy * ny + dz * nz;
                    const float rx = dx - (2.0f * dn) * nx, ry = dy - (2.0f * dn) * ny, rz = dz - (2.0f * dn) * nz;
                    const float rl = sqrtf(rx * rx + ry * ry + rz * rz);
                    dx = rx / rl;
                    dy = ry / rl;
                    dz = rz / rl;
                    ox = sox;
                    oy = soy;
                    oz = soz;
                    ++rays;
                } else {
                    cr += w * lr;
                    cg += w * lg;
                    cb += w * lb;
                    break;
                }
            }
            float *o = out + 4 * (j * width + i);
            o[0] = cr;
            o[1] = cg;
            o[2] = cb;
            o[3] = (float)rays;
        }
    }
}
