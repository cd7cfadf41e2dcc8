/*
 * FP64 CPU oracle for direct measurement-equation visibility prediction and peeling
 * (Line et al., "Modelling and peeling extended sources with shapelets", arXiv 2005.09316).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check of __graft_entry__ and the
 * cpu_baseline / reference leg of bench.py may load or call this library.  It shares no
 * code, header, table or helper with the CUDA library; the two meet only through the
 * seeded inputs of synth/.
 *
 * Everything is plain FP64 with straightforward loops, in the order the paper writes it:
 *
 *   V(u,v,w) = sum_j  S_j(nu) * xi_j(u,v) * exp(-2 pi i (u l_j + v m_j + w (n_j - 1)))
 *
 * (Sec. 3.1, eq:measure_eq_discrete, with the beam B == 1 as the paper's simulator uses it;
 *  Sec. 3.2, eq:env_visi_def for the envelope xi).  u, v, w are in wavelengths: the metres of the
 * input are scaled by nu / c per channel (Sec. 3.2, last paragraph: uvw are computed once per time
 * step and scaled by frequency).
 *
 * Readings of the paper taken here (each is listed in the design notes):
 *  - eq:basis_1D prints pi^2 in the normalisation; orthonormality (Sec. 2) needs pi^(1/2).  The
 *    uv-space envelope uses the peak-normalised Hermite functions
 *        phi_n(x) = H_n(x) exp(-x^2/2) / sqrt(2^n n!)
 *    so that B_00 reduces exactly to the Gaussian envelope when beta1 = maj, beta2 = min (Sec. 3.2).
 *  - eq:basis_FT prints i^(p1+p2); the e^{-2 pi i} kernel of eq:measure_eq gives (-i)^(p1+p2).
 *  - eq:shape-env prints p_k + p_l < p_max; the fit (Sec. 2.1) and p_tot use <=.  We use <=.
 *  - The shapelet (u, v) are re-phased to the shapelet centre (Sec. 3.2 after eq:scale-shape-y):
 *    (u', v', w') = R(H_j, dec_j) R(H_0, dec_0)^T (u, v, w); the phase term keeps u, l.
 *  - Spectrum S(nu) = S_ref (nu / nu_ref)^alpha (Sec. 4.1: a flux at 180 MHz and one spectral index).
 *  - Peel residual R_ij = D_ij - g_i conj(g_j) V_ij (Sec. 5.1).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_C_LIGHT 299792458.0
#define OR_NMAX_LIMIT 127

static const double OR_PI = 3.14159265358979323846;

/* n - 1 for a direction (l, m), with n = sqrt(1 - l^2 - m^2) (Sec. 3.1, below eq:measure_eq),
 * written as -(l^2 + m^2) / (1 + n) so that it does not cancel for small l, m. */
double or_n_minus_1(double l, double m)
{
    double r2 = l * l + m * m;
    return -r2 / (1.0 + sqrt(1.0 - r2));
}

/* Power-law spectrum (Sec. 4.1 and Sec. 6: one flux at a reference frequency and one spectral index). */
double or_spectrum(double s_ref, double alpha, double nu_ref, double nu)
{
    return s_ref * pow(nu / nu_ref, alpha);
}

/* Gaussian visibility envelope, eq:gauss-env with eq:scale-gauss-x and eq:scale-gauss-y.
 * u, v in wavelengths; maj, min are FWHM in radians; pa in radians, East of North. */
double or_gauss_env(double u, double v, double maj, double min, double pa)
{
    double kx = cos(pa) * v + sin(pa) * u;
    double ky = -sin(pa) * v + cos(pa) * u;
    double e = OR_PI * OR_PI / (4.0 * log(2.0));
    return exp(-e * (kx * kx * maj * maj + ky * ky * min * min));
}

/* Peak-normalised Hermite functions phi_0..phi_nmax at x by the three-term recurrence of the
 * Hermite polynomials (H_{n+1} = 2x H_n - 2n H_{n-1}) divided through by sqrt(2^(n+1) (n+1)!). */
void or_hermite(int nmax, double x, double* phi)
{
    phi[0] = exp(-0.5 * x * x);
    if (nmax >= 1) phi[1] = sqrt(2.0) * x * phi[0];
    for (int n = 1; n < nmax; ++n)
        phi[n + 1] = sqrt(2.0 / (n + 1)) * x * phi[n] - sqrt((double)n / (n + 1)) * phi[n - 1];
}

/* (-i)^k, the phase factor of the analytic Fourier transform (eq:basis_FT, with the sign that the
 * e^{-2 pi i} measurement equation gives). */
static double complex or_minus_i_pow(int k)
{
    switch (k & 3) {
    case 0: return 1.0;
    case 1: return -I;
    case 2: return -1.0;
    default: return I;
    }
}

/* Rotation R(H, dec) from XYZ to (u, v, w) for a phase centre at hour angle H, declination dec. */
static void or_uvw_rotation(double h, double dec, double r[9])
{
    double sh = sin(h), ch = cos(h), sd = sin(dec), cd = cos(dec);
    r[0] = sh;        r[1] = ch;        r[2] = 0.0;
    r[3] = -sd * ch;  r[4] = sd * sh;   r[5] = cd;
    r[6] = cd * ch;   r[7] = -cd * sh;  r[8] = sd;
}

/* Derivatives of R(H, dec) with respect to H and to dec (differentiating or_uvw_rotation entry by entry). */
static void or_uvw_rotation_dh(double h, double dec, double r[9])
{
    double sh = sin(h), ch = cos(h), sd = sin(dec), cd = cos(dec);
    r[0] = ch;        r[1] = -sh;       r[2] = 0.0;
    r[3] = sd * sh;   r[4] = sd * ch;   r[5] = 0.0;
    r[6] = -cd * sh;  r[7] = -cd * ch;  r[8] = 0.0;
}

static void or_uvw_rotation_ddec(double h, double dec, double r[9])
{
    double sh = sin(h), ch = cos(h), sd = sin(dec), cd = cos(dec);
    r[0] = 0.0;       r[1] = 0.0;       r[2] = 0.0;
    r[3] = -cd * ch;  r[4] = cd * sh;   r[5] = -sd;
    r[6] = -sd * ch;  r[7] = sd * sh;   r[8] = cd;
}

/* Frame that re-phases (u, v, w) from the phase centre (H0, dec0) to a shapelet centred at (l, m)
 * (Sec. 3.2, the u_{i,j}, v_{i,j} of eq:scale-shape-x/y).  The centre (RA_j, dec_j) follows from
 * (l, m) by inverting the orthographic projection: sin dec_j = m cos dec0 + n sin dec0,
 * RA_j - RA_0 = atan2(l, n cos dec0 - m sin dec0).  With H = LST - RA, H_j = H0 - (RA_j - RA_0),
 * and F = R(H_j, dec_j) R(H0, dec0)^T does not depend on H0, so H0 = 0 is used. */
void or_shapelet_frame(double l, double m, double dec0, double f[9])
{
    double n = sqrt(1.0 - l * l - m * m);
    double dec_j = asin(m * cos(dec0) + n * sin(dec0));
    double dra = atan2(l, n * cos(dec0) - m * sin(dec0));
    double rj[9], r0[9];
    or_uvw_rotation(-dra, dec_j, rj);
    or_uvw_rotation(0.0, dec0, r0);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += rj[3 * a + k] * r0[3 * b + k];
            f[3 * a + b] = s;
        }
}

/* Derivatives of that frame with respect to l and m.  The centre moves with (l, m): dec_j through
 * sin dec_j = m cos dec0 + n sin dec0 and RA_j - RA_0 = atan2(l, X), X = n cos dec0 - m sin dec0,
 * n = sqrt(1 - l^2 - m^2); with F = R(-dra, dec_j) R(0, dec0)^T the chain rule gives
 * dF/dl = (-dR/dH d(dra)/dl + dR/ddec d(dec_j)/dl) R(0, dec0)^T, and likewise for m. */
void or_shapelet_frame_grad(double l, double m, double dec0, double fl[9], double fm[9])
{
    double n = sqrt(1.0 - l * l - m * m);
    double dn_dl = -l / n, dn_dm = -m / n;
    double s = m * cos(dec0) + n * sin(dec0);
    double dec_j = asin(s), c = sqrt(1.0 - s * s);
    double ddec_dl = dn_dl * sin(dec0) / c, ddec_dm = (cos(dec0) + dn_dm * sin(dec0)) / c;
    double X = n * cos(dec0) - m * sin(dec0);
    double dX_dl = dn_dl * cos(dec0), dX_dm = dn_dm * cos(dec0) - sin(dec0);
    double dra = atan2(l, X), den = X * X + l * l;
    double ddra_dl = (X - l * dX_dl) / den, ddra_dm = -l * dX_dm / den;
    double rh[9], rd[9], r0[9];
    or_uvw_rotation_dh(-dra, dec_j, rh);
    or_uvw_rotation_ddec(-dra, dec_j, rd);
    or_uvw_rotation(0.0, dec0, r0);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double sl = 0.0, sm = 0.0;
            for (int k = 0; k < 3; ++k) {
                double gl = -rh[3 * a + k] * ddra_dl + rd[3 * a + k] * ddec_dl;
                double gm = -rh[3 * a + k] * ddra_dm + rd[3 * a + k] * ddec_dm;
                sl += gl * r0[3 * b + k];
                sm += gm * r0[3 * b + k];
            }
            fl[3 * a + b] = sl;
            fm[3 * a + b] = sm;
        }
}

/* Shapelet visibility envelope, eq:shape-env with eq:scale-shape-x/y and eq:basis_FT:
 *   xi = sum_{n1+n2<=nmax} C[n1,n2] (-i)^(n1+n2) phi_n1(beta1 kx) phi_n2(beta2 ky),
 *   kx = pi/sqrt(2 ln 2) (cos(pa) v' + sin(pa) u'),  ky = pi/sqrt(2 ln 2) (-sin(pa) v' + cos(pa) u').
 * up, vp in wavelengths in the shapelet's own frame. */
double complex or_shapelet_env(double up, double vp, double beta1, double beta2, double pa, int nmax,
                               int nnz, const int* n1, const int* n2, const double* c)
{
    double K = OR_PI / sqrt(2.0 * log(2.0));
    double kx = K * (cos(pa) * vp + sin(pa) * up);
    double ky = K * (-sin(pa) * vp + cos(pa) * up);
    double px[OR_NMAX_LIMIT + 2], py[OR_NMAX_LIMIT + 2];
    or_hermite(nmax, beta1 * kx, px);
    or_hermite(nmax, beta2 * ky, py);
    double complex xi = 0.0;
    for (int k = 0; k < nnz; ++k)
        xi += c[k] * or_minus_i_pow(n1[k] + n2[k]) * px[n1[k]] * py[n2[k]];
    return xi;
}

static void or_set_threads(int n_threads)
{
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Direct prediction (eq:env_visi_def) of n_rows rows of visibilities over n_chan channels.
 * uvw[r*3 + 0..2] in metres; vis[(r*n_chan + f)*2 + {0,1}] = (Re, Im).
 * Components: the first n_point are points (xi = 1), the next n_gauss Gaussians, the last n_shape
 * shapelets; per-component arrays l, m, s_ref, alpha, nu_ref are indexed over all of them.
 * Shapelet s uses coefficient triples s_off[s] .. s_off[s+1]-1.
 */
void or_predict(int n_rows, const double* uvw, int n_chan, const double* freq, double dec0,
                int n_point, int n_gauss, int n_shape,
                const double* l, const double* m, const double* s_ref, const double* alpha,
                const double* nu_ref, const double* g_maj, const double* g_min, const double* g_pa,
                const double* s_b1, const double* s_b2, const double* s_pa, const int* s_nmax,
                const int* s_off, const int* s_n1, const int* s_n2, const double* s_c,
                double* vis, int n_threads)
{
    int n_comp = n_point + n_gauss + n_shape;
    double* frames = (double*)malloc(sizeof(double) * 9 * (n_shape > 0 ? n_shape : 1));
    for (int s = 0; s < n_shape; ++s) {
        int j = n_point + n_gauss + s;
        or_shapelet_frame(l[j], m[j], dec0, frames + 9 * s);
    }
    or_set_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < n_rows; ++r) {
        const double* b = uvw + 3 * r;
        for (int f = 0; f < n_chan; ++f) {
            double inv_lambda = freq[f] / OR_C_LIGHT;
            double u = b[0] * inv_lambda, v = b[1] * inv_lambda, w = b[2] * inv_lambda;
            double complex sum = 0.0;
            for (int j = 0; j < n_comp; ++j) {
                double phase = u * l[j] + v * m[j] + w * or_n_minus_1(l[j], m[j]);
                double complex xi = 1.0;
                if (j >= n_point && j < n_point + n_gauss) {
                    int g = j - n_point;
                    xi = or_gauss_env(u, v, g_maj[g], g_min[g], g_pa[g]);
                } else if (j >= n_point + n_gauss) {
                    int s = j - n_point - n_gauss;
                    const double* F = frames + 9 * s;
                    double up = F[0] * u + F[1] * v + F[2] * w;
                    double vp = F[3] * u + F[4] * v + F[5] * w;
                    xi = or_shapelet_env(up, vp, s_b1[s], s_b2[s], s_pa[s], s_nmax[s], s_off[s + 1] - s_off[s],
                                         s_n1 + s_off[s], s_n2 + s_off[s], s_c + s_off[s]);
                }
                sum += or_spectrum(s_ref[j], alpha[j], nu_ref[j], freq[f]) * xi * cexp(-2.0 * OR_PI * I * phase);
            }
            vis[2 * ((size_t)r * n_chan + f) + 0] = creal(sum);
            vis[2 * ((size_t)r * n_chan + f) + 1] = cimag(sum);
        }
    }
    free(frames);
}

/*
 * Peel residual R = D - g[a1] conj(g[a2]) V (Sec. 5.1: M_ij = g_i g_j^* I_ij, R_ij = V_ij - M_ij).
 * Rows are (t, b) pairs given by row_t, row_b; gains are [n_tg][n_fg][n_ant] complex, broadcast
 * over time when n_tg == 1 and over channel when n_fg == 1.  All complex arrays interleaved.
 */
void or_peel(int n_rows, const int* row_t, const int* row_b, const int* ant1, const int* ant2,
             int n_ant, const double* gains, int n_tg, int n_fg, int n_chan,
             const double* data, const double* vis, double* resid)
{
    for (int r = 0; r < n_rows; ++r) {
        int tg = n_tg == 1 ? 0 : row_t[r];
        for (int f = 0; f < n_chan; ++f) {
            int fg = n_fg == 1 ? 0 : f;
            const double* g1 = gains + 2 * (((size_t)tg * n_fg + fg) * n_ant + ant1[row_b[r]]);
            const double* g2 = gains + 2 * (((size_t)tg * n_fg + fg) * n_ant + ant2[row_b[r]]);
            double complex G = (g1[0] + I * g1[1]) * conj(g2[0] + I * g2[1]);
            size_t k = 2 * ((size_t)r * n_chan + f);
            double complex R = (data[k] + I * data[k + 1]) - G * (vis[k] + I * vis[k + 1]);
            resid[k] = creal(R);
            resid[k + 1] = cimag(R);
        }
    }
}

/*
 * Analytic gradient of L = sum |D - G V|^2 with respect to the component parameters, given the
 * per-visibility weight W = conj(G) (D - G V) (interleaved, [n_rows][n_chan]):
 *     dL/dp = -2 sum_vis Re( conj(W) dV/dp ).
 * The paper fits in image space and gives no derivatives; they follow from differentiating
 * eq:env_visi_def term by term:
 *   dV_j/dS_ref = V_j / S_ref;  dV_j/dalpha = ln(nu/nu_ref) V_j;
 *   dV_j/dl = -2 pi i (u - w l / n) V_j  (likewise m); for a shapelet also S P dxi/dl through its
 *     re-phasing frame: dxi/dl = dxi/dx beta1 dkx/dl + dxi/dy beta2 dky/dl, with (dup/dl, dvp/dl) from
 *     or_shapelet_frame_grad (eq:scale-shape-x/y take u, v in the shapelet's own frame);
 *   Gaussian: dxi/dmaj = -2E maj kx^2 xi, dxi/dmin = -2E min ky^2 xi, dxi/dpa = -2E (maj^2-min^2) kx ky xi;
 *   Shapelet: with x = beta1 kx, y = beta2 ky and phi_n' = sqrt(n/2) phi_{n-1} - sqrt((n+1)/2) phi_{n+1},
 *     dxi/dbeta1 = sum c s phi_n1'(x) kx phi_n2(y);  dxi/dbeta2 = sum c s phi_n1(x) phi_n2'(y) ky;
 *     dxi/dpa = sum c s (phi_n1'(x) beta1 ky phi_n2(y) - phi_n1(x) phi_n2'(y) beta2 kx);
 *     dxi/dc_k = s phi_n1(x) phi_n2(y),  s = (-i)^(n1+n2).
 * Outputs are accumulated (+=) so the caller zeroes them: g_comp[n_comp * 4] holds (flux, alpha, l, m)
 * per component; g_gauss[n_gauss * 3] (maj, min, pa); g_shape[n_shape * 3] (beta1, beta2, pa);
 * g_coeff[nnz].  Single-threaded: the order of the sums is fixed.
 */
void or_grad(int n_rows, const double* uvw, int n_chan, const double* freq, double dec0,
             int n_point, int n_gauss, int n_shape,
             const double* l, const double* m, const double* s_ref, const double* alpha,
             const double* nu_ref, const double* g_maj, const double* g_min, const double* g_pa,
             const double* s_b1, const double* s_b2, const double* s_pa, const int* s_nmax,
             const int* s_off, const int* s_n1, const int* s_n2, const double* s_c,
             const double* W, double* g_comp, double* g_gauss, double* g_shape, double* g_coeff)
{
    int n_comp = n_point + n_gauss + n_shape;
    double E = OR_PI * OR_PI / (4.0 * log(2.0));
    double K = OR_PI / sqrt(2.0 * log(2.0));
    for (int r = 0; r < n_rows; ++r) {
        const double* b = uvw + 3 * r;
        for (int f = 0; f < n_chan; ++f) {
            double inv_lambda = freq[f] / OR_C_LIGHT;
            double u = b[0] * inv_lambda, v = b[1] * inv_lambda, w = b[2] * inv_lambda;
            size_t k = 2 * ((size_t)r * n_chan + f);
            double complex cw = W[k] - I * W[k + 1]; /* conj(W) */
            for (int j = 0; j < n_comp; ++j) {
                double n = sqrt(1.0 - l[j] * l[j] - m[j] * m[j]);
                double phase = u * l[j] + v * m[j] + w * or_n_minus_1(l[j], m[j]);
                double complex P = cexp(-2.0 * OR_PI * I * phase);
                double S = or_spectrum(s_ref[j], alpha[j], nu_ref[j], freq[f]);
                double complex xi = 1.0;
                if (j >= n_point && j < n_point + n_gauss) {
                    int g = j - n_point;
                    double pa = g_pa[g], mj = g_maj[g], mn = g_min[g];
                    double kx = cos(pa) * v + sin(pa) * u, ky = -sin(pa) * v + cos(pa) * u;
                    xi = or_gauss_env(u, v, mj, mn, pa);
                    double complex base = cw * S * P;
                    g_gauss[3 * g + 0] += -2.0 * creal(base * (-2.0 * E * mj * kx * kx * xi));
                    g_gauss[3 * g + 1] += -2.0 * creal(base * (-2.0 * E * mn * ky * ky * xi));
                    g_gauss[3 * g + 2] += -2.0 * creal(base * (-2.0 * E * (mj * mj - mn * mn) * kx * ky * xi));
                } else if (j >= n_point + n_gauss) {
                    int s = j - n_point - n_gauss;
                    double F[9];
                    or_shapelet_frame(l[j], m[j], dec0, F);
                    double up = F[0] * u + F[1] * v + F[2] * w;
                    double vp = F[3] * u + F[4] * v + F[5] * w;
                    double pa = s_pa[s], b1 = s_b1[s], b2 = s_b2[s];
                    double kx = K * (cos(pa) * vp + sin(pa) * up);
                    double ky = K * (-sin(pa) * vp + cos(pa) * up);
                    int nmax = s_nmax[s];
                    double px[OR_NMAX_LIMIT + 3], py[OR_NMAX_LIMIT + 3], dx[OR_NMAX_LIMIT + 2], dy[OR_NMAX_LIMIT + 2];
                    or_hermite(nmax + 1, b1 * kx, px);
                    or_hermite(nmax + 1, b2 * ky, py);
                    for (int q = 0; q <= nmax; ++q) {
                        dx[q] = (q > 0 ? sqrt(q / 2.0) * px[q - 1] : 0.0) - sqrt((q + 1) / 2.0) * px[q + 1];
                        dy[q] = (q > 0 ? sqrt(q / 2.0) * py[q - 1] : 0.0) - sqrt((q + 1) / 2.0) * py[q + 1];
                    }
                    double complex dxi_b1 = 0.0, dxi_b2 = 0.0, dxi_pa = 0.0, dxi_x = 0.0, dxi_y = 0.0;
                    xi = 0.0;
                    double complex base = cw * S * P;
                    for (int q = s_off[s]; q < s_off[s + 1]; ++q) {
                        int a = s_n1[q], c2 = s_n2[q];
                        double complex ph = or_minus_i_pow(a + c2);
                        xi += s_c[q] * ph * px[a] * py[c2];
                        dxi_x += s_c[q] * ph * dx[a] * py[c2];
                        dxi_y += s_c[q] * ph * px[a] * dy[c2];
                        dxi_b1 += s_c[q] * ph * dx[a] * kx * py[c2];
                        dxi_b2 += s_c[q] * ph * px[a] * dy[c2] * ky;
                        dxi_pa += s_c[q] * ph * (dx[a] * b1 * ky * py[c2] - px[a] * dy[c2] * b2 * kx);
                        g_coeff[q] += -2.0 * creal(base * ph * px[a] * py[c2]);
                    }
                    g_shape[3 * s + 0] += -2.0 * creal(base * dxi_b1);
                    g_shape[3 * s + 1] += -2.0 * creal(base * dxi_b2);
                    g_shape[3 * s + 2] += -2.0 * creal(base * dxi_pa);
                    /* the position moves the frame: (up, vp) and so (x, y) depend on (l, m) */
                    double Fl[9], Fm[9];
                    or_shapelet_frame_grad(l[j], m[j], dec0, Fl, Fm);
                    double dup_l = Fl[0] * u + Fl[1] * v + Fl[2] * w, dvp_l = Fl[3] * u + Fl[4] * v + Fl[5] * w;
                    double dup_m = Fm[0] * u + Fm[1] * v + Fm[2] * w, dvp_m = Fm[3] * u + Fm[4] * v + Fm[5] * w;
                    double dkx_l = K * (cos(pa) * dvp_l + sin(pa) * dup_l), dky_l = K * (-sin(pa) * dvp_l + cos(pa) * dup_l);
                    double dkx_m = K * (cos(pa) * dvp_m + sin(pa) * dup_m), dky_m = K * (-sin(pa) * dvp_m + cos(pa) * dup_m);
                    g_comp[4 * j + 2] += -2.0 * creal(base * (dxi_x * b1 * dkx_l + dxi_y * b2 * dky_l));
                    g_comp[4 * j + 3] += -2.0 * creal(base * (dxi_x * b1 * dkx_m + dxi_y * b2 * dky_m));
                }
                double complex Vj = S * xi * P;
                double complex t = cw * Vj;
                g_comp[4 * j + 0] += -2.0 * creal(t) / s_ref[j];
                g_comp[4 * j + 1] += -2.0 * creal(t) * log(freq[f] / nu_ref[j]);
                g_comp[4 * j + 2] += -2.0 * creal(t * (-2.0 * OR_PI * I) * (u - w * l[j] / n));
                g_comp[4 * j + 3] += -2.0 * creal(t * (-2.0 * OR_PI * I) * (v - w * m[j] / n));
            }
        }
    }
}
