/*
 * FP64 CPU oracle for the D3Q19 variant of the two-component MRT
 * pseudopotential lattice Boltzmann step with corrected open boundaries.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow restatement of the
 * method in three dimensions that the CUDA D3Q19 path is checked against.
 * Only the test suite, the smoke check and the benchmark's CPU legs may load
 * it.  It shares no code, header, table or helper with the CUDA library.
 *
 * The paper runs 3D cases (Sec. III C, Fig. 8; Sec. III D, Figs. 10-11) but
 * prints only the 2D operators.  This oracle carries every 2D stage over to
 * 3D, the readings being:
 *   - lattice: D3Q19, rest / 6 face / 12 edge velocities with weights 1/3,
 *     1/18, 1/36 (c_s^2 = 1/3);
 *   - collision: Eq. 1 with dense 19x19 T, S, T^-1; T is the orthogonal
 *     19-moment basis (rho, e, eps, j_x, q_x, j_y, q_y, j_z, q_z, 3p_xx,
 *     3pi_xx, p_ww, pi_ww, p_xy, p_yz, p_xz, m_x, m_y, m_z) built from its
 *     moment polynomials; S = diag[1, s_e, s_eps, 1, s_q, 1, s_q, 1, s_q,
 *     s_nu, s_pi, s_nu, s_pi, s_nu, s_nu, s_nu, s_m, s_m, s_m] with
 *     s_pi = s_eps and s_m = s_q (the paper is silent on the 3D-only
 *     rates);
 *   - equilibrium Eq. 6, forcing Eq. 9, macroscopic fields Eqs. 7-8 with
 *     three velocity components;
 *   - forces Eqs. 10-11 on the 92-vector 8th-order isotropic 3D stencil
 *     (|e|^2 in {1,2,3,4,5,6,8}); its weights are NOT printed and are
 *     obtained here at start-up by solving the isotropy conditions (second
 *     moment 1 as for the printed 2D weights; isotropic 4th, 6th and 8th
 *     moments) with Gaussian elimination;
 *   - open faces: Eq. 13 NEQ extrapolation over the 5 unknowns (the
 *     directions with e.n < 0, n the outward normal), the alpha correction
 *     of Eqs. 15-19 with three components, alpha_i = w_i sum_a e_ia D_a /
 *     sum_U e_a^2 w; Eqs. 20-23 at the outlet with lambda and chi averaged
 *     over the face; Eqs. 24-25 mirrored across every open side;
 *   - halfway bounce-back Eq. B1 and periodic wrap Eq. B2 on each axis.
 * The step order is that of the D2Q9 oracle (stream, inlet, outlet, rho,
 * forces, u^eq with chi, collision, lagged lambda/chi reductions).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q3 19
#define NC 2
#define NST 92

static const int EX3[Q3] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int EY3[Q3] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int EZ3[Q3] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1};
static const double CS2 = 1.0 / 3.0;

static double w3(int i) {
    int e2 = EX3[i] * EX3[i] + EY3[i] * EY3[i] + EZ3[i] * EZ3[i];
    if (e2 == 0) return 1.0 / 3.0;
    if (e2 == 1) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

static int opp3(int i) {
    for (int j = 0; j < Q3; ++j)
        if (EX3[j] == -EX3[i] && EY3[j] == -EY3[i] && EZ3[j] == -EZ3[i]) return j;
    return -1;
}

static double T3[Q3][Q3], T3inv[Q3][Q3];
static int SX[NST], SY[NST], SZ[NST];
static double SW[NST];
static double shell_w[9]; /* weight per |e|^2 */
static int ready3 = 0;

/* Solve the n x n system A x = b in place (partial pivoting). */
static int gauss(int n, double* A, double* b) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
        if (fabs(A[piv * n + c]) < 1e-300) return -1;
        if (piv != c) {
            for (int k = 0; k < n; ++k) {
                double t = A[c * n + k];
                A[c * n + k] = A[piv * n + k];
                A[piv * n + k] = t;
            }
            double t = b[c];
            b[c] = b[piv];
            b[piv] = t;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double m = A[r * n + c] / A[c * n + c];
            for (int k = c; k < n; ++k) A[r * n + k] -= m * A[c * n + k];
            b[r] -= m * b[c];
        }
    }
    for (int c = 0; c < n; ++c) b[c] /= A[c * n + c];
    return 0;
}

/* sum over the vectors of shell r2 (|e|^2 = r2, components in [-2, 2]) of
 * e_x^a e_y^b e_z^c */
static double shell_moment(int r2, int a, int b, int c) {
    double s = 0.0;
    for (int z = -2; z <= 2; ++z)
        for (int y = -2; y <= 2; ++y)
            for (int x = -2; x <= 2; ++x) {
                if (x * x + y * y + z * z != r2) continue;
                s += pow(x, a) * pow(y, b) * pow(z, c);
            }
    return s;
}

/* Weights of the 8th-order isotropic 3D stencil: unknown w(r2) for
 * r2 in {1,2,3,4,5,6,8}; conditions (M_abc = sum w e_x^a e_y^b e_z^c):
 *   M_200 = 1;  M_400 = 3 M_220;  M_600 = 5 M_420;  M_420 = 3 M_222;
 *   M_800 = 7 M_620;  9 M_620 = 15 M_440;  M_440 = 3 M_422
 * (the ratios of the isotropic tensors delta^(4), delta^(6), delta^(8)). */
static void solve_shell_weights(void) {
    static const int R2[7] = {1, 2, 3, 4, 5, 6, 8};
    double A[49], b[7] = {1, 0, 0, 0, 0, 0, 0};
    for (int j = 0; j < 7; ++j) {
        int r = R2[j];
        A[0 * 7 + j] = shell_moment(r, 2, 0, 0);
        A[1 * 7 + j] = shell_moment(r, 4, 0, 0) - 3.0 * shell_moment(r, 2, 2, 0);
        A[2 * 7 + j] = shell_moment(r, 6, 0, 0) - 5.0 * shell_moment(r, 4, 2, 0);
        A[3 * 7 + j] = shell_moment(r, 4, 2, 0) - 3.0 * shell_moment(r, 2, 2, 2);
        A[4 * 7 + j] = shell_moment(r, 8, 0, 0) - 7.0 * shell_moment(r, 6, 2, 0);
        A[5 * 7 + j] = 9.0 * shell_moment(r, 6, 2, 0) - 15.0 * shell_moment(r, 4, 4, 0);
        A[6 * 7 + j] = shell_moment(r, 4, 4, 0) - 3.0 * shell_moment(r, 4, 2, 2);
    }
    gauss(7, A, b);
    for (int r = 0; r < 9; ++r) shell_w[r] = 0.0;
    for (int j = 0; j < 7; ++j) shell_w[R2[j]] = b[j];
}

static void build3(void) {
    if (ready3) return;
    for (int i = 0; i < Q3; ++i) {
        double ex = EX3[i], ey = EY3[i], ez = EZ3[i];
        double e2 = ex * ex + ey * ey + ez * ez;
        double r[Q3] = {
            1.0,
            19.0 * e2 - 30.0,
            (21.0 * e2 * e2 - 53.0 * e2 + 24.0) / 2.0,
            ex, (5.0 * e2 - 9.0) * ex,
            ey, (5.0 * e2 - 9.0) * ey,
            ez, (5.0 * e2 - 9.0) * ez,
            3.0 * ex * ex - e2, (3.0 * e2 - 5.0) * (3.0 * ex * ex - e2),
            ey * ey - ez * ez, (3.0 * e2 - 5.0) * (ey * ey - ez * ez),
            ex * ey, ey * ez, ex * ez,
            (ey * ey - ez * ez) * ex, (ez * ez - ex * ex) * ey, (ex * ex - ey * ey) * ez};
        for (int m = 0; m < Q3; ++m) T3[m][i] = r[m];
    }
    /* rows are mutually orthogonal: T^-1 = T^T diag(1/|row|^2) */
    for (int m = 0; m < Q3; ++m) {
        double nrm = 0.0;
        for (int i = 0; i < Q3; ++i) nrm += T3[m][i] * T3[m][i];
        for (int i = 0; i < Q3; ++i) T3inv[i][m] = T3[m][i] / nrm;
    }
    solve_shell_weights();
    int c = 0;
    for (int z = -2; z <= 2; ++z)
        for (int y = -2; y <= 2; ++y)
            for (int x = -2; x <= 2; ++x) {
                int r2 = x * x + y * y + z * z;
                if (r2 == 0 || r2 > 8 || shell_w[r2] == 0.0) continue;
                SX[c] = x;
                SY[c] = y;
                SZ[c] = z;
                SW[c] = shell_w[r2];
                ++c;
            }
    ready3 = 1;
}

/* Eq. 6 in 3D */
void orc3_feq(double rho, double ux, double uy, double uz, double* out) {
    double uu = ux * ux + uy * uy + uz * uz;
    for (int i = 0; i < Q3; ++i) {
        double eu = EX3[i] * ux + EY3[i] * uy + EZ3[i] * uz;
        out[i] = rho * w3(i) * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

/* Eq. 9 in 3D */
void orc3_fbar(double ux, double uy, double uz, double Fx, double Fy, double Fz, double* out) {
    for (int i = 0; i < Q3; ++i) {
        double ex = EX3[i], ey = EY3[i], ez = EZ3[i];
        double eu = ex * ux + ey * uy + ez * uz;
        double ax = (ex - ux) / CS2 + eu * ex / (CS2 * CS2);
        double ay = (ey - uy) / CS2 + eu * ey / (CS2 * CS2);
        double az = (ez - uz) / CS2 + eu * ez / (CS2 * CS2);
        out[i] = w3(i) * (ax * Fx + ay * Fy + az * Fz);
    }
}

/* Eq. 1 for one component at one node (dense 19x19 transforms). */
void orc3_collide(const double* f, double rho, const double* u, const double* F, const double* s,
                  double* out) {
    build3();
    double feq[Q3], fb[Q3], m[Q3], mf[Q3], g[Q3];
    orc3_feq(rho, u[0], u[1], u[2], feq);
    orc3_fbar(u[0], u[1], u[2], F[0], F[1], F[2], fb);
    for (int r = 0; r < Q3; ++r) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < Q3; ++i) {
            a += T3[r][i] * (f[i] - feq[i]);
            b += T3[r][i] * fb[i];
        }
        m[r] = a;
        mf[r] = b;
    }
    for (int r = 0; r < Q3; ++r) g[r] = -s[r] * m[r] + (1.0 - 0.5 * s[r]) * mf[r];
    for (int i = 0; i < Q3; ++i) {
        double a = 0.0;
        for (int r = 0; r < Q3; ++r) a += T3inv[i][r] * g[r];
        out[i] = f[i] + a;
    }
}

void orc3_moment_matrix(double* T, double* Tinv) {
    build3();
    for (int r = 0; r < Q3; ++r)
        for (int c = 0; c < Q3; ++c) {
            if (T) T[r * Q3 + c] = T3[r][c];
            if (Tinv) Tinv[r * Q3 + c] = T3inv[r][c];
        }
}

void orc3_lattice(int* ex, int* ey, int* ez, double* w, int* opp) {
    for (int i = 0; i < Q3; ++i) {
        if (ex) ex[i] = EX3[i];
        if (ey) ey[i] = EY3[i];
        if (ez) ez[i] = EZ3[i];
        if (w) w[i] = w3(i);
        if (opp) opp[i] = opp3(i);
    }
}

int orc3_stencil(int* dx, int* dy, int* dz, double* w) {
    build3();
    for (int c = 0; c < NST; ++c) {
        if (dx) dx[c] = SX[c];
        if (dy) dy[c] = SY[c];
        if (dz) dz[c] = SZ[c];
        if (w) w[c] = SW[c];
    }
    return NST;
}

/* ---------------------------------------------------------------------- */
typedef struct {
    int nx, ny, nz;
    int periodic[3];
    double G12;
    double Gw[2];
    double nu[2];
    double s_e;     /* > 0: shared s_e; <= 0: s_e,k = s_nu,k */
    double s_q;     /* q and m rates */
    int s_eps_mode; /* 1: s_eps (and s_pi) from max nu; 0: own nu_k */
    double body[3];
} orc3_params;

typedef struct {
    int kind;         /* 1 velocity inlet, 2 convective outlet */
    int side;         /* 0 x=0, 1 x=nx-1, 2 y=0, 3 y=ny-1, 4 z=0, 5 z=nz-1 */
    int lo[2], hi[2]; /* inclusive extent on the tangential axes (first: the lower axis) */
    double rho_in[2];
    int alpha_on, chi_on;
} orc3_face;

#define MAXF3 6

typedef struct {
    orc3_params p;
    int nfaces;
    orc3_face face[MAXF3];
    double* prof[MAXF3];  /* inward normal speed per face position */
    double* rprof[MAXF3]; /* [2][len] composition per face position */
    int nx, ny, nz;
    long N;
    uint8_t* solid;
    int* faceid;
    double s[2][Q3];
    double *f, *fpost, *fpost_prev, *rho, *u, *F, *Fprev;
    double lambda, chi, Qin, Qout, Umean;
    long step;
    int threads;
} orc3_state;

#define F3(k, i, n) ((((size_t)(k)) * Q3 + (i)) * (size_t)N + (size_t)(n))

static void normal3(int side, int* o) {
    o[0] = o[1] = o[2] = 0;
    o[side / 2] = (side & 1) ? 1 : -1;
}

/* tangential axes of a side: the two axes other than side/2, ascending */
static void tangential(int side, int* a0, int* a1) {
    int ax = side / 2;
    *a0 = ax == 0 ? 1 : 0;
    *a1 = ax == 2 ? 1 : 2;
}

static int face_len(const orc3_face* fc, int* l0) {
    *l0 = fc->hi[0] - fc->lo[0] + 1;
    return *l0 * (fc->hi[1] - fc->lo[1] + 1);
}

/* coordinates of face position (t0, t1) */
static void face_xyz(const orc3_state* st, const orc3_face* fc, int t0, int t1, int* c) {
    int ext[3] = {st->nx, st->ny, st->nz};
    int a0, a1, ax = fc->side / 2;
    tangential(fc->side, &a0, &a1);
    c[ax] = (fc->side & 1) ? ext[ax] - 1 : 0;
    c[a0] = t0;
    c[a1] = t1;
}

static int open_side(const orc3_state* st, int side) {
    for (int f = 0; f < st->nfaces; ++f)
        if (st->face[f].side == side) return 1;
    return 0;
}

static long idx3(const orc3_state* st, const int* c) {
    return ((long)c[2] * st->ny + c[1]) * st->nx + c[0];
}

/* psi / solid-indicator site (Eqs. 10, 11, 24, 25): 1 = solid */
static int psi_site3(const orc3_state* st, int x, int y, int z, long* n) {
    int c[3] = {x, y, z}, ext[3] = {st->nx, st->ny, st->nz};
    for (int a = 0; a < 3; ++a) {
        if (c[a] >= 0 && c[a] < ext[a]) continue;
        if (st->p.periodic[a]) c[a] = ((c[a] % ext[a]) + ext[a]) % ext[a];
        else if (c[a] < 0 && open_side(st, 2 * a)) c[a] = -1 - c[a];
        else if (c[a] >= ext[a] && open_side(st, 2 * a + 1)) c[a] = 2 * ext[a] - 1 - c[a];
        else return 1;
    }
    *n = idx3(st, c);
    return st->solid[*n] ? 1 : 0;
}

/* pull source (Eq. 2): 1 = blocked (bounce-back or open-face unknown) */
static int pull_site3(const orc3_state* st, int x, int y, int z, long* n) {
    int c[3] = {x, y, z}, ext[3] = {st->nx, st->ny, st->nz};
    for (int a = 0; a < 3; ++a) {
        if (c[a] >= 0 && c[a] < ext[a]) continue;
        if (!st->p.periodic[a]) return 1;
        c[a] = ((c[a] % ext[a]) + ext[a]) % ext[a];
    }
    *n = idx3(st, c);
    return st->solid[*n] ? 1 : 0;
}

void orc3_destroy(orc3_state* st) {
    if (!st) return;
    free(st->solid);
    free(st->faceid);
    free(st->f);
    free(st->fpost);
    free(st->fpost_prev);
    free(st->rho);
    free(st->u);
    free(st->F);
    free(st->Fprev);
    for (int f = 0; f < MAXF3; ++f) {
        free(st->prof[f]);
        free(st->rprof[f]);
    }
    free(st);
}

static void derive_rates3(orc3_state* st) {
    const orc3_params* p = &st->p;
    double numax = p->nu[0] > p->nu[1] ? p->nu[0] : p->nu[1];
    for (int k = 0; k < NC; ++k) {
        double snu = 1.0 / (3.0 * p->nu[k] + 0.5);
        double seps = p->s_eps_mode ? 1.0 / (3.0 * numax + 0.5) : snu;
        double se = p->s_e > 0.0 ? p->s_e : snu;
        double sq = p->s_q;
        double s[Q3] = {1.0, se, seps, 1.0, sq, 1.0, sq, 1.0, sq, snu, seps, snu, seps, snu, snu, snu, sq, sq, sq};
        for (int r = 0; r < Q3; ++r) st->s[k][r] = s[r];
    }
}

/* profiles[f]: normal speed per face position (may be NULL = 0);
 * rprofiles[f]: [2][len] composition (NULL = rho_in). */
orc3_state* orc3_create(const orc3_params* p, int nfaces, const orc3_face* faces, const double* const* profiles,
                        const double* const* rprofiles, const uint8_t* solid, const double* rho_init,
                        const double* u_init) {
    build3();
    if (!p || p->nx < 5 || p->ny < 5 || p->nz < 5 || nfaces < 0 || nfaces > MAXF3) return NULL;
    orc3_state* st = (orc3_state*)calloc(1, sizeof(orc3_state));
    if (!st) return NULL;
    st->p = *p;
    st->nx = p->nx;
    st->ny = p->ny;
    st->nz = p->nz;
    st->N = (long)p->nx * p->ny * p->nz;
    long N = st->N;
    st->threads = 1;
    st->solid = (uint8_t*)calloc((size_t)N, 1);
    st->faceid = (int*)calloc((size_t)N, sizeof(int));
    size_t nf = (size_t)NC * Q3 * N;
    st->f = (double*)calloc(nf, sizeof(double));
    st->fpost = (double*)calloc(nf, sizeof(double));
    st->fpost_prev = (double*)calloc(nf, sizeof(double));
    st->rho = (double*)calloc((size_t)NC * N, sizeof(double));
    st->u = (double*)calloc((size_t)3 * N, sizeof(double));
    st->F = (double*)calloc((size_t)NC * 3 * N, sizeof(double));
    st->Fprev = (double*)calloc((size_t)NC * 3 * N, sizeof(double));
    if (!st->solid || !st->faceid || !st->f || !st->fpost || !st->fpost_prev || !st->rho || !st->u || !st->F ||
        !st->Fprev) {
        orc3_destroy(st);
        return NULL;
    }
    if (solid)
        for (long n = 0; n < N; ++n) st->solid[n] = solid[n] ? 1 : 0;
    int ext[3] = {st->nx, st->ny, st->nz};
    int nout = 0;
    st->nfaces = nfaces;
    for (int f = 0; f < nfaces; ++f) {
        orc3_face fc = faces[f];
        st->face[f] = fc;
        if (fc.kind != 1 && fc.kind != 2) goto bad;
        if (fc.side < 0 || fc.side > 5 || p->periodic[fc.side / 2]) goto bad;
        int a0, a1;
        tangential(fc.side, &a0, &a1);
        if (fc.lo[0] < 0 || fc.hi[0] >= ext[a0] || fc.lo[0] > fc.hi[0]) goto bad;
        if (fc.lo[1] < 0 || fc.hi[1] >= ext[a1] || fc.lo[1] > fc.hi[1]) goto bad;
        if (fc.kind == 2) ++nout;
        int l0, len = face_len(&fc, &l0);
        st->prof[f] = (double*)calloc((size_t)len, sizeof(double));
        st->rprof[f] = (double*)calloc((size_t)2 * len, sizeof(double));
        if (!st->prof[f] || !st->rprof[f]) goto bad;
        if (profiles && profiles[f]) memcpy(st->prof[f], profiles[f], (size_t)len * sizeof(double));
        for (int q = 0; q < len; ++q)
            for (int k = 0; k < 2; ++k)
                st->rprof[f][(size_t)k * len + q] =
                    (rprofiles && rprofiles[f]) ? rprofiles[f][(size_t)k * len + q] : fc.rho_in[k];
        for (int t1 = fc.lo[1]; t1 <= fc.hi[1]; ++t1)
            for (int t0 = fc.lo[0]; t0 <= fc.hi[0]; ++t0) {
                int c[3];
                face_xyz(st, &fc, t0, t1, c);
                long n = idx3(st, c);
                if (st->solid[n]) continue;
                if (st->faceid[n]) goto bad;
                st->faceid[n] = f + 1;
            }
    }
    if (nout > 1) goto bad;
    for (int f = 0; f < nfaces; ++f) {
        const orc3_face* fc = &st->face[f];
        int o[3];
        normal3(fc->side, o);
        for (int t1 = fc->lo[1]; t1 <= fc->hi[1]; ++t1)
            for (int t0 = fc->lo[0]; t0 <= fc->hi[0]; ++t0) {
                int c[3];
                face_xyz(st, fc, t0, t1, c);
                long n = idx3(st, c);
                if (st->solid[n]) continue;
                int c2[3] = {c[0] - o[0], c[1] - o[1], c[2] - o[2]};
                long n2 = idx3(st, c2);
                if (st->solid[n2] || st->faceid[n2]) goto bad;
            }
    }
    derive_rates3(st);
    for (long n = 0; n < N; ++n) {
        if (st->solid[n]) continue;
        double uu[3];
        for (int a = 0; a < 3; ++a) {
            uu[a] = u_init ? u_init[(size_t)a * N + n] : 0.0;
            st->u[(size_t)a * N + n] = uu[a];
        }
        for (int k = 0; k < NC; ++k) {
            double feq[Q3];
            double r = rho_init[(size_t)k * N + n];
            st->rho[(size_t)k * N + n] = r;
            orc3_feq(r, uu[0], uu[1], uu[2], feq);
            for (int i = 0; i < Q3; ++i) st->f[F3(k, i, n)] = feq[i];
        }
    }
    memcpy(st->fpost, st->f, sizeof(double) * nf);
    memcpy(st->fpost_prev, st->f, sizeof(double) * nf);
    st->lambda = 0.0;
    st->chi = 1.0;
    return st;
bad:
    orc3_destroy(st);
    return NULL;
}

void orc3_set_threads(orc3_state* st, int threads) { st->threads = threads > 0 ? threads : 1; }

static void step3(orc3_state* st) {
    const int nx = st->nx, ny = st->ny, nz = st->nz;
    const long N = st->N;
    double* f = st->f;
    double* fp = st->fpost;
    int nth = st->threads;
    (void)nth;
    memcpy(st->fpost_prev, st->fpost, sizeof(double) * NC * Q3 * (size_t)N);
    memcpy(st->Fprev, st->F, sizeof(double) * NC * 3 * (size_t)N);

    /* 1. streaming (Eq. 2) with bounce-back (Eq. B1) and periodic wrap (Eq. B2) */
#pragma omp parallel for schedule(static) num_threads(nth)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long n = ((long)z * ny + y) * nx + x;
                if (st->solid[n]) {
                    for (int k = 0; k < NC; ++k)
                        for (int i = 0; i < Q3; ++i) fp[F3(k, i, n)] = 0.0;
                    continue;
                }
                for (int i = 0; i < Q3; ++i) {
                    long ns;
                    int blocked = pull_site3(st, x - EX3[i], y - EY3[i], z - EZ3[i], &ns);
                    for (int k = 0; k < NC; ++k)
                        fp[F3(k, i, n)] = blocked ? f[F3(k, opp3(i), n)] : f[F3(k, i, ns)];
                }
            }

    /* 2. inlets: Eq. 13 over the 5 unknowns, then Eqs. 15-19 */
    for (int fi = 0; fi < st->nfaces; ++fi) {
        const orc3_face* fc = &st->face[fi];
        if (fc->kind != 1) continue;
        int o[3];
        normal3(fc->side, o);
        int U[Q3], nu = 0;
        double sa[3] = {0, 0, 0};
        for (int i = 0; i < Q3; ++i)
            if (EX3[i] * o[0] + EY3[i] * o[1] + EZ3[i] * o[2] < 0) {
                U[nu++] = i;
                sa[0] += EX3[i] * EX3[i] * w3(i);
                sa[1] += EY3[i] * EY3[i] * w3(i);
                sa[2] += EZ3[i] * EZ3[i] * w3(i);
            }
        int l0, len = face_len(fc, &l0);
        for (int t1 = fc->lo[1]; t1 <= fc->hi[1]; ++t1)
            for (int t0 = fc->lo[0]; t0 <= fc->hi[0]; ++t0) {
                int c[3];
                face_xyz(st, fc, t0, t1, c);
                long n1 = idx3(st, c);
                if (st->solid[n1]) continue;
                int c2[3] = {c[0] - o[0], c[1] - o[1], c[2] - o[2]};
                long n2 = idx3(st, c2);
                int q = (t1 - fc->lo[1]) * l0 + (t0 - fc->lo[0]);
                double speed = st->prof[fi][q];
                double uin[3] = {-o[0] * speed, -o[1] * speed, -o[2] * speed};
                double rin[2] = {st->rprof[fi][q], st->rprof[fi][(size_t)len + q]};
                double rho2[NC], j[3] = {0, 0, 0};
                for (int k = 0; k < NC; ++k) {
                    rho2[k] = 0.0;
                    for (int i = 0; i < Q3; ++i) {
                        double v = fp[F3(k, i, n2)];
                        rho2[k] += v;
                        j[0] += EX3[i] * v;
                        j[1] += EY3[i] * v;
                        j[2] += EZ3[i] * v;
                    }
                    for (int a = 0; a < 3; ++a) j[a] += 0.5 * st->Fprev[((size_t)k * 3 + a) * N + n2];
                }
                double u2[3];
                for (int a = 0; a < 3; ++a) u2[a] = j[a] / (rho2[0] + rho2[1]);
                for (int k = 0; k < NC; ++k) {
                    double feq1[Q3], feq2[Q3];
                    orc3_feq(rin[k], uin[0], uin[1], uin[2], feq1);
                    orc3_feq(rho2[k], u2[0], u2[1], u2[2], feq2);
                    for (int a = 0; a < nu; ++a) {
                        int i = U[a];
                        fp[F3(k, i, n1)] = feq1[i] + (fp[F3(k, i, n2)] - feq2[i]);
                    }
                    if (fc->alpha_on) {
                        double mom[3];
                        for (int a = 0; a < 3; ++a) mom[a] = 0.5 * st->Fprev[((size_t)k * 3 + a) * N + n1];
                        for (int i = 0; i < Q3; ++i) {
                            mom[0] += EX3[i] * fp[F3(k, i, n1)];
                            mom[1] += EY3[i] * fp[F3(k, i, n1)];
                            mom[2] += EZ3[i] * fp[F3(k, i, n1)];
                        }
                        double d[3];
                        for (int a = 0; a < 3; ++a) d[a] = rin[k] * uin[a] - mom[a];
                        for (int a = 0; a < nu; ++a) {
                            int i = U[a];
                            double al = w3(i) * (EX3[i] * d[0] / sa[0] + EY3[i] * d[1] / sa[1] + EZ3[i] * d[2] / sa[2]);
                            fp[F3(k, i, n1)] += al;
                        }
                    }
                }
            }
    }

    /* 3. outlet: Eq. 20 with lambda of the previous step */
    for (int fi = 0; fi < st->nfaces; ++fi) {
        const orc3_face* fc = &st->face[fi];
        if (fc->kind != 2) continue;
        int o[3];
        normal3(fc->side, o);
        for (int t1 = fc->lo[1]; t1 <= fc->hi[1]; ++t1)
            for (int t0 = fc->lo[0]; t0 <= fc->hi[0]; ++t0) {
                int c[3];
                face_xyz(st, fc, t0, t1, c);
                long nN = idx3(st, c);
                if (st->solid[nN]) continue;
                int c2[3] = {c[0] - o[0], c[1] - o[1], c[2] - o[2]};
                long nN1 = idx3(st, c2);
                for (int i = 0; i < Q3; ++i) {
                    if (EX3[i] * o[0] + EY3[i] * o[1] + EZ3[i] * o[2] >= 0) continue;
                    for (int k = 0; k < NC; ++k)
                        fp[F3(k, i, nN)] = (st->fpost_prev[F3(k, i, nN)] + st->lambda * fp[F3(k, i, nN1)]) /
                                           (1.0 + st->lambda);
                }
            }
    }

    /* 4. densities, psi_k = rho_k */
    double* rho = st->rho;
#pragma omp parallel for schedule(static) num_threads(nth)
    for (long n = 0; n < N; ++n)
        for (int k = 0; k < NC; ++k) {
            double r = 0.0;
            if (!st->solid[n])
                for (int i = 0; i < Q3; ++i) r += fp[F3(k, i, n)];
            rho[(size_t)k * N + n] = r;
        }

    /* 5. forces (Eqs. 10, 11) + body force; 6. u^eq (Eqs. 7, 8) */
    double* F = st->F;
    double* u = st->u;
#pragma omp parallel for schedule(static) num_threads(nth)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long n = ((long)z * ny + y) * nx + x;
                if (st->solid[n]) {
                    for (int q = 0; q < 6; ++q) F[(size_t)q * N + n] = 0.0;
                    for (int a = 0; a < 3; ++a) u[(size_t)a * N + n] = 0.0;
                    continue;
                }
                double g[NC][3] = {{0, 0, 0}, {0, 0, 0}}, ad[3] = {0, 0, 0};
                for (int c = 0; c < NST; ++c) {
                    long m;
                    int e[3] = {SX[c], SY[c], SZ[c]};
                    if (psi_site3(st, x + e[0], y + e[1], z + e[2], &m)) {
                        for (int a = 0; a < 3; ++a) ad[a] += SW[c] * e[a];
                    } else {
                        for (int k = 0; k < NC; ++k)
                            for (int a = 0; a < 3; ++a) g[k][a] += SW[c] * rho[(size_t)k * N + m] * e[a];
                    }
                }
                double rt = rho[n] + rho[N + n];
                double j[3] = {0, 0, 0};
                for (int k = 0; k < NC; ++k) {
                    double pk = rho[(size_t)k * N + n];
                    for (int a = 0; a < 3; ++a) {
                        double Fa = -st->p.G12 * pk * g[1 - k][a] - st->p.Gw[k] * pk * ad[a] + st->p.body[a] * pk / rt;
                        F[((size_t)k * 3 + a) * N + n] = Fa;
                        j[a] += 0.5 * Fa;
                    }
                    for (int i = 0; i < Q3; ++i) {
                        double v = fp[F3(k, i, n)];
                        j[0] += EX3[i] * v;
                        j[1] += EY3[i] * v;
                        j[2] += EZ3[i] * v;
                    }
                }
                for (int a = 0; a < 3; ++a) u[(size_t)a * N + n] = j[a] / rt;
            }

    /* Eq. 22: outlet normal velocity = chi * that of the inward neighbour */
    for (int fi = 0; fi < st->nfaces; ++fi) {
        const orc3_face* fc = &st->face[fi];
        if (fc->kind != 2 || !fc->chi_on) continue;
        int o[3], ax = fc->side / 2;
        normal3(fc->side, o);
        for (int t1 = fc->lo[1]; t1 <= fc->hi[1]; ++t1)
            for (int t0 = fc->lo[0]; t0 <= fc->hi[0]; ++t0) {
                int c[3];
                face_xyz(st, fc, t0, t1, c);
                long nN = idx3(st, c);
                if (st->solid[nN]) continue;
                int c2[3] = {c[0] - o[0], c[1] - o[1], c[2] - o[2]};
                long nN1 = idx3(st, c2);
                u[(size_t)ax * N + nN] = st->chi * u[(size_t)ax * N + nN1];
            }
    }

    /* 7. collision (Eq. 1) */
#pragma omp parallel for schedule(static) num_threads(nth)
    for (long n = 0; n < N; ++n) {
        if (st->solid[n]) {
            for (int k = 0; k < NC; ++k)
                for (int i = 0; i < Q3; ++i) f[F3(k, i, n)] = 0.0;
            continue;
        }
        double un[3] = {u[n], u[N + n], u[2 * N + n]};
        for (int k = 0; k < NC; ++k) {
            double fin[Q3], fo[Q3], Fk[3];
            for (int i = 0; i < Q3; ++i) fin[i] = fp[F3(k, i, n)];
            for (int a = 0; a < 3; ++a) Fk[a] = F[((size_t)k * 3 + a) * N + n];
            orc3_collide(fin, rho[(size_t)k * N + n], un, Fk, st->s[k], fo);
            for (int i = 0; i < Q3; ++i) f[F3(k, i, n)] = fo[i];
        }
    }

    /* 8. lagged reductions for lambda (Eq. 21) and chi (Eq. 23) */
    double qin = 0.0, qout = 0.0, usum = 0.0;
    int have_in = 0, have_out = 0;
    long mcount = 0;
    for (int fi = 0; fi < st->nfaces; ++fi) {
        const orc3_face* fc = &st->face[fi];
        int o[3], ax = fc->side / 2;
        normal3(fc->side, o);
        double sgn = (fc->side & 1) ? 1.0 : -1.0;
        for (int t1 = fc->lo[1]; t1 <= fc->hi[1]; ++t1)
            for (int t0 = fc->lo[0]; t0 <= fc->hi[0]; ++t0) {
                int c[3];
                face_xyz(st, fc, t0, t1, c);
                long n1 = idx3(st, c);
                if (st->solid[n1]) continue;
                if (fc->kind == 1) {
                    have_in = 1;
                    qin += (rho[n1] + rho[N + n1]) * (-sgn * u[(size_t)ax * N + n1]);
                } else {
                    have_out = 1;
                    int c2[3] = {c[0] - o[0], c[1] - o[1], c[2] - o[2]};
                    long n2 = idx3(st, c2);
                    double un = sgn * u[(size_t)ax * N + n2];
                    qout += (rho[n2] + rho[N + n2]) * un;
                    usum += un;
                    ++mcount;
                }
            }
    }
    st->Qin = qin;
    st->Qout = qout;
    if (have_out && mcount > 0) {
        double lam = usum / mcount;
        st->Umean = lam;
        st->lambda = lam > 0.0 ? lam : 0.0;
        st->chi = (!have_in || fabs(qout) < 1e-14) ? 1.0 : qin / qout;
    }
    st->step += 1;
}

void orc3_step(orc3_state* st, int nsteps) {
    for (int s = 0; s < nsteps; ++s) step3(st);
}

void orc3_get_macros(const orc3_state* st, double* rho, double* u, double* F) {
    size_t N = (size_t)st->N;
    if (rho) memcpy(rho, st->rho, sizeof(double) * 2 * N);
    if (u) memcpy(u, st->u, sizeof(double) * 3 * N);
    if (F) memcpy(F, st->F, sizeof(double) * 6 * N);
}

void orc3_get_f(const orc3_state* st, double* f) {
    memcpy(f, st->f, sizeof(double) * NC * Q3 * (size_t)st->N);
}

/* Post-stream, post-boundary populations of the last step, [2][19][N]. */
void orc3_get_fpost(const orc3_state* st, double* f) {
    memcpy(f, st->fpost, sizeof(double) * NC * Q3 * (size_t)st->N);
}

/* Forces of the step before the last one, [2][3][N]. */
void orc3_get_force_prev(const orc3_state* st, double* F) {
    memcpy(F, st->Fprev, sizeof(double) * NC * 3 * (size_t)st->N);
}

void orc3_set_f(orc3_state* st, const double* f) {
    memcpy(st->f, f, sizeof(double) * NC * Q3 * (size_t)st->N);
}

/* out: [lambda, chi, Qin, Qout, Umean, mass_1, mass_2, step, s(2x19)...] */
void orc3_get_scalars(const orc3_state* st, double* out) {
    double m[NC] = {0.0, 0.0};
    size_t N = (size_t)st->N;
    for (int k = 0; k < NC; ++k)
        for (size_t n = 0; n < N; ++n)
            if (!st->solid[n])
                for (int i = 0; i < Q3; ++i) m[k] += st->f[F3(k, i, n)];
    out[0] = st->lambda;
    out[1] = st->chi;
    out[2] = st->Qin;
    out[3] = st->Qout;
    out[4] = st->Umean;
    out[5] = m[0];
    out[6] = m[1];
    out[7] = (double)st->step;
    for (int k = 0; k < NC; ++k)
        for (int r = 0; r < Q3; ++r) out[8 + k * Q3 + r] = st->s[k][r];
}

/* Forces of Eqs. 10/11 for given psi [2][N] on the state's geometry: F [2][3][N]. */
void orc3_eval_forces(const orc3_state* st, const double* psi, double* F) {
    long N = st->N;
    for (int z = 0; z < st->nz; ++z)
        for (int y = 0; y < st->ny; ++y)
            for (int x = 0; x < st->nx; ++x) {
                long n = ((long)z * st->ny + y) * st->nx + x;
                double g[2][3] = {{0, 0, 0}, {0, 0, 0}}, ad[3] = {0, 0, 0};
                if (!st->solid[n])
                    for (int c = 0; c < NST; ++c) {
                        long m;
                        int e[3] = {SX[c], SY[c], SZ[c]};
                        if (psi_site3(st, x + e[0], y + e[1], z + e[2], &m)) {
                            for (int a = 0; a < 3; ++a) ad[a] += SW[c] * e[a];
                        } else
                            for (int k = 0; k < 2; ++k)
                                for (int a = 0; a < 3; ++a) g[k][a] += SW[c] * psi[(size_t)k * N + m] * e[a];
                    }
                for (int k = 0; k < 2; ++k) {
                    double pk = st->solid[n] ? 0.0 : psi[(size_t)k * N + n];
                    for (int a = 0; a < 3; ++a)
                        F[((size_t)k * 3 + a) * N + n] = -st->p.G12 * pk * g[1 - k][a] - st->p.Gw[k] * pk * ad[a];
                }
            }
}
