/*
 * FP64 CPU oracle for the two-component MRT pseudopotential lattice Boltzmann
 * step with the corrected open boundaries (D2Q9).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * restatement of the method that the CUDA path is checked against.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Every stage follows the paper in its own order and notation:
 *   - lattice: D2Q9 velocities e_0..e_8 and weights omega_i (Sec. II A, after
 *     Eq. 6); the velocity order is fixed by the unknown sets {1,5,8},
 *     {3,6,7}, {4,7,8} of Eqs. 13, 14, 20 and App. B, Eq. B2;
 *   - collision: Eq. 1 with the dense 9x9 matrices T, S, T^-1 (Eqs. 3, 4);
 *     T is built row by row from its moment polynomials (the printed
 *     rows 3-8 of Eq. 3 are garbled, see the oracle header in oracle.py);
 *   - viscosity: Eq. 5, nu_k = (1/s_nu - 1/2)/3;
 *   - s_eps from the most viscous phase (Sec. III A);
 *   - equilibrium: Eq. 6 (quadratic term over 2 c_s^4);
 *   - macroscopic fields: Eqs. 7, 8;
 *   - forcing term: Eq. 9;
 *   - forces: Eq. 10 (fluid-fluid, 8th-order isotropic weights w(1)=4/21,
 *     w(2)=4/45, w(4)=1/60, w(5)=2/315, w(8)=1/5040), Eq. 11 (adhesion),
 *     psi_k = rho_k;
 *   - streaming: Eq. 2 (pull form), halfway bounce-back Eq. B1, periodic
 *     wrap Eq. B2;
 *   - inlet: NEQ extrapolation Eqs. 13/14, then the alpha correction
 *     Eqs. 15-19;
 *   - outlet: convective scheme Eqs. 20/21 and the mass-flux correction
 *     chi, Eqs. 22/23;
 *   - ghost layers that mirror densities across open faces, Eqs. 24/25.
 * Readings where the text is silent or garbled are listed in oracle.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NQ 9
#define NCOMP 2

/* D2Q9 velocities (Sec. II A; order fixed by Eqs. 13, 14, 20, B2). */
static const int EXV[NQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EYV[NQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double CS2 = 1.0 / 3.0; /* c_s = 1/sqrt(3) */

static double omega_of(int i) {
    int e2 = EXV[i] * EXV[i] + EYV[i] * EYV[i];
    if (e2 == 0) return 4.0 / 9.0;
    if (e2 == 1) return 1.0 / 9.0;
    return 1.0 / 36.0;
}

static int opposite_of(int i) {
    for (int j = 0; j < NQ; ++j)
        if (EXV[j] == -EXV[i] && EYV[j] == -EYV[i]) return j;
    return -1;
}

/* ---------------------------------------------------------------------- */
/* Moment matrix T (Eq. 3), built from its moment polynomials:            */
/* rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy (the order of S, Eq. 4).   */
/* ---------------------------------------------------------------------- */
static double T_mat[NQ][NQ];
static double Tinv_mat[NQ][NQ];
static int tables_ready = 0;

/* 24-point 8th-order isotropic stencil (Eq. 10, weights after Eq. 12). */
static int ST_DX[24], ST_DY[24];
static double ST_W[24];

static double weight_of_norm2(int r2) {
    switch (r2) {
    case 1: return 4.0 / 21.0;
    case 2: return 4.0 / 45.0;
    case 4: return 1.0 / 60.0;
    case 5: return 2.0 / 315.0;
    case 8: return 1.0 / 5040.0;
    default: return 0.0;
    }
}

static void build_tables(void) {
    if (tables_ready) return;
    for (int i = 0; i < NQ; ++i) {
        double ex = EXV[i], ey = EYV[i];
        double e2 = ex * ex + ey * ey;
        T_mat[0][i] = 1.0;
        T_mat[1][i] = -4.0 + 3.0 * e2;
        T_mat[2][i] = 4.0 - 10.5 * e2 + 4.5 * e2 * e2;
        T_mat[3][i] = ex;
        T_mat[4][i] = (-5.0 + 3.0 * e2) * ex;
        T_mat[5][i] = ey;
        T_mat[6][i] = (-5.0 + 3.0 * e2) * ey;
        T_mat[7][i] = ex * ex - ey * ey;
        T_mat[8][i] = ex * ey;
    }
    /* rows are mutually orthogonal, so T^-1 = T^T diag(1/|row|^2) */
    for (int r = 0; r < NQ; ++r) {
        double nrm = 0.0;
        for (int i = 0; i < NQ; ++i) nrm += T_mat[r][i] * T_mat[r][i];
        for (int i = 0; i < NQ; ++i) Tinv_mat[i][r] = T_mat[r][i] / nrm;
    }
    int c = 0;
    for (int dy = -2; dy <= 2; ++dy)
        for (int dx = -2; dx <= 2; ++dx) {
            double w = weight_of_norm2(dx * dx + dy * dy);
            if (w == 0.0) continue;
            ST_DX[c] = dx;
            ST_DY[c] = dy;
            ST_W[c] = w;
            ++c;
        }
    tables_ready = 1;
}

static void matvec(const double A[NQ][NQ], const double* x, double* y) {
    for (int r = 0; r < NQ; ++r) {
        double acc = 0.0;
        for (int c = 0; c < NQ; ++c) acc += A[r][c] * x[c];
        y[r] = acc;
    }
}

/* Eq. 6 (quadratic term read as (e.u)^2 / (2 c_s^4)). */
void orc_feq(double rho, double ux, double uy, double* out) {
    double uu = ux * ux + uy * uy;
    for (int i = 0; i < NQ; ++i) {
        double eu = EXV[i] * ux + EYV[i] * uy;
        out[i] = rho * omega_of(i) *
                 (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

/* Eq. 9: Fbar_i = omega_i [ (e_i - u)/c_s^2 + (e_i.u) e_i / c_s^4 ] . F */
void orc_fbar(double ux, double uy, double Fx, double Fy, double* out) {
    for (int i = 0; i < NQ; ++i) {
        double ex = EXV[i], ey = EYV[i];
        double eu = ex * ux + ey * uy;
        double ax = (ex - ux) / CS2 + eu * ex / (CS2 * CS2);
        double ay = (ey - uy) / CS2 + eu * ey / (CS2 * CS2);
        out[i] = omega_of(i) * (ax * Fx + ay * Fy);
    }
}

/* Eq. 1 for one component at one node:
 * f* = f - T^-1 S T (f - feq) + T^-1 (I - S/2) T Fbar. */
void orc_collide(const double* f, double rho, double ux, double uy, double Fx,
                 double Fy, const double* s, double* out) {
    build_tables();
    double feq[NQ], fb[NQ], d[NQ], m[NQ], mf[NQ], g[NQ], back[NQ];
    orc_feq(rho, ux, uy, feq);
    orc_fbar(ux, uy, Fx, Fy, fb);
    for (int i = 0; i < NQ; ++i) d[i] = f[i] - feq[i];
    matvec((const double(*)[NQ])T_mat, d, m);
    matvec((const double(*)[NQ])T_mat, fb, mf);
    for (int r = 0; r < NQ; ++r) g[r] = -s[r] * m[r] + (1.0 - 0.5 * s[r]) * mf[r];
    matvec((const double(*)[NQ])Tinv_mat, g, back);
    for (int i = 0; i < NQ; ++i) out[i] = f[i] + back[i];
}

void orc_moment_matrix(double* T, double* Tinv) {
    build_tables();
    for (int r = 0; r < NQ; ++r)
        for (int c = 0; c < NQ; ++c) {
            if (T) T[r * NQ + c] = T_mat[r][c];
            if (Tinv) Tinv[r * NQ + c] = Tinv_mat[r][c];
        }
}

void orc_lattice(int* ex, int* ey, double* w, int* opp) {
    for (int i = 0; i < NQ; ++i) {
        if (ex) ex[i] = EXV[i];
        if (ey) ey[i] = EYV[i];
        if (w) w[i] = omega_of(i);
        if (opp) opp[i] = opposite_of(i);
    }
}

int orc_stencil(int* dx, int* dy, double* w) {
    build_tables();
    for (int c = 0; c < 24; ++c) {
        if (dx) dx[c] = ST_DX[c];
        if (dy) dy[c] = ST_DY[c];
        if (w) w[c] = ST_W[c];
    }
    return 24;
}

/* ---------------------------------------------------------------------- */
/* Configuration and state                                                 */
/* ---------------------------------------------------------------------- */
typedef struct {
    int nx, ny;
    int periodic_x, periodic_y;
    double G12;
    double Gw[2];
    double nu[2];
    double s_e;       /* > 0: this s_e for both components; <= 0: s_e,k = s_nu,k */
    double s_q;       /* rate shared by q_x and q_y */
    int s_eps_mode;   /* 1: s_eps from max(nu) (Sec. III A); 0: from own nu_k */
    double body[2];   /* body-force density, shared by rho_k / rho */
    int use_s_full;   /* 1: S taken verbatim from s_full (textbook reductions) */
    double s_full[2][NQ];
    int chi_same_step; /* 1: chi of Eq. 23 from this step's fields (t + dt, as printed); 0: lagged */
    double wall_ux[2];  /* x-velocity of the walls beyond the closed edges y = 0 and y = ny-1 */
    int wet_interp;     /* 1: Eq. 12's phase-dependent adhesion coefficient (reading below) */
    double wet_delta;   /* its delta */
} orc_params;

typedef struct {
    int kind;         /* 1 = velocity inlet, 2 = convective outlet */
    int side;         /* 0: x=0, 1: x=nx-1, 2: y=0, 3: y=ny-1 */
    int lo, hi;       /* inclusive extent along the face */
    double rho_in[2]; /* prescribed component densities (inlet) */
    int alpha_on;     /* Eqs. 15-19 on/off (inlet) */
    int chi_on;       /* Eqs. 22-23 on/off (outlet) */
} orc_face;

#define MAXFACE 4

typedef struct {
    orc_params p;
    int nfaces;
    orc_face face[MAXFACE];
    double* prof[MAXFACE]; /* inward normal speed per face position */
    int nx, ny, N;
    uint8_t* solid;
    int* faceid;   /* 0: none, f+1: node belongs to face f */
    double s[2][NQ];
    double* f;          /* [2][9][N] post-collision populations f* */
    double* fpost;      /* [2][9][N] post-stream, post-BC populations of the last step */
    double* fpost_prev; /* same, one step earlier (outlet Eq. 20) */
    double* rho;        /* [2][N] */
    double* u;          /* [2][N] common velocity u^eq used by the collision */
    double* F;          /* [2][2][N] total force per component */
    double* Fprev;      /* forces of the previous step (inlet, Eqs. 13, 16) */
    double lambda, chi; /* outlet coefficients used by the next step */
    double Qin, Qout, Umean;
    long step;
    int threads;
} orc_state;

static void side_normal(int side, int* nx_out, int* ny_out) {
    /* outward normal of the face */
    *nx_out = 0;
    *ny_out = 0;
    if (side == 0) *nx_out = -1;
    if (side == 1) *nx_out = 1;
    if (side == 2) *ny_out = -1;
    if (side == 3) *ny_out = 1;
}

static void face_node(const orc_state* st, const orc_face* fc, int t, int* x, int* y) {
    if (fc->side == 0) { *x = 0; *y = t; }
    else if (fc->side == 1) { *x = st->nx - 1; *y = t; }
    else if (fc->side == 2) { *x = t; *y = 0; }
    else { *x = t; *y = st->ny - 1; }
}

static void derive_rates(orc_state* st) {
    const orc_params* p = &st->p;
    if (p->use_s_full) {
        for (int k = 0; k < NCOMP; ++k)
            for (int r = 0; r < NQ; ++r) st->s[k][r] = p->s_full[k][r];
        return;
    }
    double numax = p->nu[0] > p->nu[1] ? p->nu[0] : p->nu[1];
    for (int k = 0; k < NCOMP; ++k) {
        double snu = 1.0 / (3.0 * p->nu[k] + 0.5); /* Eq. 5 solved for s_nu */
        double seps = p->s_eps_mode ? 1.0 / (3.0 * numax + 0.5) : snu;
        double se = p->s_e > 0.0 ? p->s_e : snu;
        /* Eq. 4: diag[s_rho, s_e, s_eps, s_j, s_q, s_j, s_q, s_nu, s_nu], s_rho = s_j = 1 */
        double s[NQ] = {1.0, se, seps, 1.0, p->s_q, 1.0, p->s_q, snu, snu};
        for (int r = 0; r < NQ; ++r) st->s[k][r] = s[r];
    }
}

static int face_on_side(const orc_state* st, int side) {
    for (int f = 0; f < st->nfaces; ++f)
        if (st->face[f].side == side) return 1;
    return 0;
}

/* Eq. 12: the adhesion coefficient of both components at a node whose phase
 * indicator is rho_e = (rho_1 - rho_2)/(rho_1 + rho_2): G_w,1 beyond delta
 * (fluid 1), G_w,2 below -delta (fluid 2), and between them the two linear
 * pieces g1 = G_w,1 rho_e/delta on (0, delta] and g2 = -G_w,2 rho_e/delta on
 * (-delta, 0], which meet at 0 on the interface.  Without wet_interp each
 * component keeps its own constant G_w,k. */
static double adhesion_coeff(const orc_state* st, int k, double r1, double r2) {
    if (!st->p.wet_interp) return st->p.Gw[k];
    const double re = (r1 - r2) / (r1 + r2), d = st->p.wet_delta;
    if (re > d) return st->p.Gw[0];
    if (re > 0.0) return st->p.Gw[0] * re / d;
    if (re > -d) return -st->p.Gw[1] * re / d;
    return st->p.Gw[1];
}

/* Virtual site for the psi / solid-indicator stencil (Eqs. 10, 11, 24, 25).
 * Returns 1 when the site is solid (psi = 0, s = 1); otherwise sets *n. */
static int psi_site(const orc_state* st, int x, int y, int* n) {
    int nx = st->nx, ny = st->ny;
    if (x < 0 || x >= nx) {
        if (st->p.periodic_x) x = ((x % nx) + nx) % nx;
        else if (x < 0 && face_on_side(st, 0)) x = -1 - x;
        else if (x >= nx && face_on_side(st, 1)) x = 2 * nx - 1 - x;
        else return 1;
    }
    if (y < 0 || y >= ny) {
        if (st->p.periodic_y) y = ((y % ny) + ny) % ny;
        else if (y < 0 && face_on_side(st, 2)) y = -1 - y;
        else if (y >= ny && face_on_side(st, 3)) y = 2 * ny - 1 - y;
        else return 1;
    }
    *n = y * nx + x;
    return st->solid[*n] ? 1 : 0;
}

/* Source of a pull (Eq. 2).  Returns 1 when the source is solid or outside
 * a non-periodic edge (then bounce-back, Eq. B1, or an open-face unknown). */
static int pull_site(const orc_state* st, int x, int y, int* n) {
    int nx = st->nx, ny = st->ny;
    if (x < 0 || x >= nx) {
        if (!st->p.periodic_x) return 1;
        x = ((x % nx) + nx) % nx;
    }
    if (y < 0 || y >= ny) {
        if (!st->p.periodic_y) return 1;
        y = ((y % ny) + ny) % ny;
    }
    *n = y * nx + x;
    return st->solid[*n] ? 1 : 0;
}

#define FIDX(k, i, n) ((((size_t)(k)) * NQ + (i)) * (size_t)N + (size_t)(n))

void orc_destroy(orc_state* st) {
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
    for (int f = 0; f < MAXFACE; ++f) free(st->prof[f]);
    free(st);
}

/* Returns NULL on an invalid configuration. */
orc_state* orc_create(const orc_params* p, int nfaces, const orc_face* faces,
                      const double* const* profiles, const uint8_t* solid,
                      const double* rho_init, const double* u_init) {
    build_tables();
    if (!p || p->nx < 5 || p->ny < 5 || nfaces < 0 || nfaces > MAXFACE) return NULL;
    orc_state* st = (orc_state*)calloc(1, sizeof(orc_state));
    if (!st) return NULL;
    st->p = *p;
    st->nx = p->nx;
    st->ny = p->ny;
    st->N = p->nx * p->ny;
    int N = st->N;
    st->threads = 1;
    st->solid = (uint8_t*)calloc((size_t)N, 1);
    st->faceid = (int*)calloc((size_t)N, sizeof(int));
    st->f = (double*)calloc((size_t)NCOMP * NQ * N, sizeof(double));
    st->fpost = (double*)calloc((size_t)NCOMP * NQ * N, sizeof(double));
    st->fpost_prev = (double*)calloc((size_t)NCOMP * NQ * N, sizeof(double));
    st->rho = (double*)calloc((size_t)NCOMP * N, sizeof(double));
    st->u = (double*)calloc((size_t)2 * N, sizeof(double));
    st->F = (double*)calloc((size_t)NCOMP * 2 * N, sizeof(double));
    st->Fprev = (double*)calloc((size_t)NCOMP * 2 * N, sizeof(double));
    if (!st->solid || !st->faceid || !st->f || !st->fpost || !st->fpost_prev ||
        !st->rho || !st->u || !st->F || !st->Fprev) {
        orc_destroy(st);
        return NULL;
    }
    if (solid) memcpy(st->solid, solid, (size_t)N);
    for (int n = 0; n < N; ++n) st->solid[n] = st->solid[n] ? 1 : 0;

    int noutlet = 0;
    st->nfaces = nfaces;
    for (int f = 0; f < nfaces; ++f) {
        orc_face fc = faces[f];
        st->face[f] = fc;
        int along = (fc.side <= 1) ? st->ny : st->nx;
        if (fc.kind != 1 && fc.kind != 2) goto bad;
        if (fc.side < 0 || fc.side > 3 || fc.lo < 0 || fc.hi >= along || fc.lo > fc.hi) goto bad;
        if ((fc.side <= 1 && p->periodic_x) || (fc.side >= 2 && p->periodic_y)) goto bad;
        if (fc.kind == 2) ++noutlet;
        int len = fc.hi - fc.lo + 1;
        st->prof[f] = (double*)calloc((size_t)len, sizeof(double));
        if (!st->prof[f]) goto bad;
        if (fc.kind == 1 && profiles && profiles[f])
            memcpy(st->prof[f], profiles[f], (size_t)len * sizeof(double));
        for (int t = fc.lo; t <= fc.hi; ++t) {
            int x, y;
            face_node(st, &fc, t, &x, &y);
            int n = y * st->nx + x;
            if (st->solid[n]) continue;
            if (st->faceid[n]) goto bad; /* a node on two faces */
            st->faceid[n] = f + 1;
        }
    }
    if (noutlet > 1) goto bad;
    /* the inward neighbour of every face node must be an ordinary fluid node */
    for (int f = 0; f < nfaces; ++f) {
        const orc_face* fc = &st->face[f];
        int ox, oy;
        side_normal(fc->side, &ox, &oy);
        for (int t = fc->lo; t <= fc->hi; ++t) {
            int x, y;
            face_node(st, fc, t, &x, &y);
            int n = y * st->nx + x;
            if (st->solid[n]) continue;
            int n2 = (y - oy) * st->nx + (x - ox);
            if (st->solid[n2] || st->faceid[n2]) goto bad;
        }
    }
    derive_rates(st);

    /* initial populations: f = feq(rho_k, u) (Eq. 6) */
    for (int n = 0; n < N; ++n) {
        if (st->solid[n]) continue;
        double ux = u_init ? u_init[n] : 0.0;
        double uy = u_init ? u_init[N + n] : 0.0;
        st->u[n] = ux;
        st->u[N + n] = uy;
        for (int k = 0; k < NCOMP; ++k) {
            double feq[NQ];
            double r = rho_init[(size_t)k * N + n];
            st->rho[(size_t)k * N + n] = r;
            orc_feq(r, ux, uy, feq);
            for (int i = 0; i < NQ; ++i) st->f[FIDX(k, i, n)] = feq[i];
        }
    }
    memcpy(st->fpost_prev, st->f, sizeof(double) * NCOMP * NQ * (size_t)N);
    memcpy(st->fpost, st->f, sizeof(double) * NCOMP * NQ * (size_t)N);
    st->lambda = 0.0;
    st->chi = 1.0;
    st->step = 0;
    return st;
bad:
    orc_destroy(st);
    return NULL;
}

void orc_set_threads(orc_state* st, int threads) {
    st->threads = threads > 0 ? threads : 1;
}

/* Mass fluxes of Eqs. 21 and 23 over the current fields: Q_in at the inlet
 * nodes x1, Q_out and the normal-speed sum at the outlet's inward neighbours
 * x_{N-1} (count in *m).  Returns 1 if the domain has an outlet. */
static int face_fluxes(const orc_state* st, double* qin, double* qout, double* usum, int* m, int* have_in) {
    const int nx = st->nx, N = st->N;
    const double* rho = st->rho;
    const double* u = st->u;
    int have_out = 0;
    *qin = *qout = *usum = 0.0;
    *m = 0;
    *have_in = 0;
    for (int fi = 0; fi < st->nfaces; ++fi) {
        const orc_face* fc = &st->face[fi];
        int ox, oy;
        side_normal(fc->side, &ox, &oy);
        for (int t = fc->lo; t <= fc->hi; ++t) {
            int x, y;
            face_node(st, fc, t, &x, &y);
            int n1 = y * nx + x;
            if (st->solid[n1]) continue;
            if (fc->kind == 1) {
                *have_in = 1;
                double un = -(ox * u[n1] + oy * u[N + n1]);
                *qin += (rho[n1] + rho[N + n1]) * un;
            } else {
                have_out = 1;
                int n2 = (y - oy) * nx + (x - ox);
                double un = ox * u[n2] + oy * u[N + n2];
                *qout += (rho[n2] + rho[N + n2]) * un;
                *usum += un;
                *m += 1;
            }
        }
    }
    return have_out;
}

/* One full time step in the canonical order:
 * stream + bounce-back + periodic -> inlet (Eq. 13, alpha) -> outlet (Eq. 20)
 * -> rho, psi, ghosts -> forces -> u^eq (chi at the outlet) -> collision
 * -> lagged reductions for lambda and chi. */
static void one_step(orc_state* st) {
    const int nx = st->nx, ny = st->ny, N = st->N;
    double* f = st->f;
    double* fp = st->fpost;
    int nth = st->threads;
    (void)nth;

    /* previous-stage copies used by the open boundaries */
    memcpy(st->fpost_prev, st->fpost, sizeof(double) * NCOMP * NQ * (size_t)N);
    memcpy(st->Fprev, st->F, sizeof(double) * NCOMP * 2 * (size_t)N);
    int opp[NQ];
    for (int i = 0; i < NQ; ++i) opp[i] = opposite_of(i);

    /* 1. streaming (Eq. 2), bounce-back (Eq. B1), periodic wrap (Eq. B2) */
#pragma omp parallel for schedule(static) num_threads(nth)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int n = y * nx + x;
            if (st->solid[n]) {
                for (int k = 0; k < NCOMP; ++k)
                    for (int i = 0; i < NQ; ++i) fp[FIDX(k, i, n)] = 0.0;
                continue;
            }
            for (int i = 0; i < NQ; ++i) {
                int ns;
                int blocked = pull_site(st, x - EXV[i], y - EYV[i], &ns);
                for (int k = 0; k < NCOMP; ++k)
                    fp[FIDX(k, i, n)] = blocked ? f[FIDX(k, opp[i], n)] : f[FIDX(k, i, ns)];
                /* moving wall beyond a closed y edge (halfway bounce-back with
                 * the wall's momentum): f_i += 2 w_i rho_k (e_i . u_w) / c_s^2,
                 * rho_k the node's own density (its post-collision sum) */
                const int sy = y - EYV[i];
                if (blocked && !st->p.periodic_y && (sy < 0 || sy >= ny)) {
                    const double uw = st->p.wall_ux[sy < 0 ? 0 : 1];
                    if (uw != 0.0)
                        for (int k = 0; k < NCOMP; ++k) {
                            double rk = 0.0;
                            for (int j = 0; j < NQ; ++j) rk += f[FIDX(k, j, n)];
                            fp[FIDX(k, i, n)] += 2.0 * omega_of(i) * rk * (EXV[i] * uw) / CS2;
                        }
                }
            }
        }

    /* 2. inlets: Eq. 13 (Eq. 14 for a vertical face), then Eqs. 15-19 */
    for (int fi = 0; fi < st->nfaces; ++fi) {
        const orc_face* fc = &st->face[fi];
        if (fc->kind != 1) continue;
        int ox, oy;
        side_normal(fc->side, &ox, &oy);
        int U[NQ], nu = 0;
        double sxx = 0.0, syy = 0.0;
        for (int i = 0; i < NQ; ++i)
            if (EXV[i] * ox + EYV[i] * oy < 0) {
                U[nu++] = i;
                sxx += EXV[i] * EXV[i] * omega_of(i);
                syy += EYV[i] * EYV[i] * omega_of(i);
            }
        for (int t = fc->lo; t <= fc->hi; ++t) {
            int x, y;
            face_node(st, fc, t, &x, &y);
            int n1 = y * nx + x;
            if (st->solid[n1]) continue;
            int n2 = (y - oy) * nx + (x - ox);
            double speed = st->prof[fi][t - fc->lo];
            double uin_x = -ox * speed, uin_y = -oy * speed;
            /* macroscopic state at x2 from its post-stream populations */
            double rho2[NCOMP], jx = 0.0, jy = 0.0;
            for (int k = 0; k < NCOMP; ++k) {
                rho2[k] = 0.0;
                for (int i = 0; i < NQ; ++i) {
                    double v = fp[FIDX(k, i, n2)];
                    rho2[k] += v;
                    jx += EXV[i] * v;
                    jy += EYV[i] * v;
                }
                jx += 0.5 * st->Fprev[((size_t)k * 2 + 0) * N + n2];
                jy += 0.5 * st->Fprev[((size_t)k * 2 + 1) * N + n2];
            }
            double u2x = jx / (rho2[0] + rho2[1]);
            double u2y = jy / (rho2[0] + rho2[1]);
            for (int k = 0; k < NCOMP; ++k) {
                double feq1[NQ], feq2[NQ];
                orc_feq(fc->rho_in[k], uin_x, uin_y, feq1);
                orc_feq(rho2[k], u2x, u2y, feq2);
                for (int a = 0; a < nu; ++a) {
                    int i = U[a];
                    fp[FIDX(k, i, n1)] = feq1[i] + (fp[FIDX(k, i, n2)] - feq2[i]);
                }
                if (fc->alpha_on) {
                    double mx = 0.5 * st->Fprev[((size_t)k * 2 + 0) * N + n1];
                    double my = 0.5 * st->Fprev[((size_t)k * 2 + 1) * N + n1];
                    for (int i = 0; i < NQ; ++i) {
                        mx += EXV[i] * fp[FIDX(k, i, n1)];
                        my += EYV[i] * fp[FIDX(k, i, n1)];
                    }
                    double dx = fc->rho_in[k] * uin_x - mx;
                    double dy = fc->rho_in[k] * uin_y - my;
                    for (int a = 0; a < nu; ++a) {
                        int i = U[a];
                        double alpha = omega_of(i) * (EXV[i] * dx / sxx + EYV[i] * dy / syy);
                        fp[FIDX(k, i, n1)] += alpha;
                    }
                }
            }
        }
    }

    /* 3. outlet: Eq. 20 with lambda of the previous step */
    for (int fi = 0; fi < st->nfaces; ++fi) {
        const orc_face* fc = &st->face[fi];
        if (fc->kind != 2) continue;
        int ox, oy;
        side_normal(fc->side, &ox, &oy);
        for (int t = fc->lo; t <= fc->hi; ++t) {
            int x, y;
            face_node(st, fc, t, &x, &y);
            int nN = y * nx + x;
            if (st->solid[nN]) continue;
            int nN1 = (y - oy) * nx + (x - ox);
            for (int i = 0; i < NQ; ++i) {
                if (EXV[i] * ox + EYV[i] * oy >= 0) continue;
                for (int k = 0; k < NCOMP; ++k)
                    fp[FIDX(k, i, nN)] =
                        (st->fpost_prev[FIDX(k, i, nN)] + st->lambda * fp[FIDX(k, i, nN1)]) /
                        (1.0 + st->lambda);
            }
        }
    }

    /* 4. densities, psi_k = rho_k */
    double* rho = st->rho;
#pragma omp parallel for schedule(static) num_threads(nth)
    for (int n = 0; n < N; ++n)
        for (int k = 0; k < NCOMP; ++k) {
            double r = 0.0;
            if (!st->solid[n])
                for (int i = 0; i < NQ; ++i) r += fp[FIDX(k, i, n)];
            rho[(size_t)k * N + n] = r;
        }

    /* 5. forces (Eqs. 10, 11) + body force; 6. common velocity (Eqs. 7, 8) */
    double* F = st->F;
    double* u = st->u;
#pragma omp parallel for schedule(static) num_threads(nth)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int n = y * nx + x;
            if (st->solid[n]) {
                for (int q = 0; q < 4; ++q) F[(size_t)q * N + n] = 0.0;
                u[n] = 0.0;
                u[N + n] = 0.0;
                continue;
            }
            double gx[NCOMP] = {0.0, 0.0}, gy[NCOMP] = {0.0, 0.0};
            double ax = 0.0, ay = 0.0;
            for (int c = 0; c < 24; ++c) {
                int m;
                int sol = psi_site(st, x + ST_DX[c], y + ST_DY[c], &m);
                if (sol) {
                    ax += ST_W[c] * ST_DX[c];
                    ay += ST_W[c] * ST_DY[c];
                } else {
                    for (int k = 0; k < NCOMP; ++k) {
                        gx[k] += ST_W[c] * rho[(size_t)k * N + m] * ST_DX[c];
                        gy[k] += ST_W[c] * rho[(size_t)k * N + m] * ST_DY[c];
                    }
                }
            }
            double rt = rho[n] + rho[N + n];
            double jx = 0.0, jy = 0.0;
            for (int k = 0; k < NCOMP; ++k) {
                int kb = 1 - k; /* the other component */
                double psik = rho[(size_t)k * N + n];
                const double gw = adhesion_coeff(st, k, rho[n], rho[N + n]);
                double Fx = -st->p.G12 * psik * gx[kb] - gw * psik * ax +
                            st->p.body[0] * psik / rt;
                double Fy = -st->p.G12 * psik * gy[kb] - gw * psik * ay +
                            st->p.body[1] * psik / rt;
                F[((size_t)k * 2 + 0) * N + n] = Fx;
                F[((size_t)k * 2 + 1) * N + n] = Fy;
                for (int i = 0; i < NQ; ++i) {
                    jx += EXV[i] * fp[FIDX(k, i, n)];
                    jy += EYV[i] * fp[FIDX(k, i, n)];
                }
                jx += 0.5 * Fx;
                jy += 0.5 * Fy;
            }
            u[n] = jx / rt;
            u[N + n] = jy / rt;
        }

    /* Eq. 23 as printed (t + dt): chi from this step's velocities, before
     * Eq. 22 uses it (lambda stays lagged: Eq. 20 needs it before the
     * velocities of this step exist) */
    if (st->p.chi_same_step) {
        double qi, qo, us;
        int mm, hin;
        if (face_fluxes(st, &qi, &qo, &us, &mm, &hin) && mm > 0)
            st->chi = (!hin || fabs(qo) < 1e-14) ? 1.0 : qi / qo;
    }

    /* Eq. 22: outlet normal velocity = chi * that of the node x_{N-1} */
    for (int fi = 0; fi < st->nfaces; ++fi) {
        const orc_face* fc = &st->face[fi];
        if (fc->kind != 2 || !fc->chi_on) continue;
        int ox, oy;
        side_normal(fc->side, &ox, &oy);
        for (int t = fc->lo; t <= fc->hi; ++t) {
            int x, y;
            face_node(st, fc, t, &x, &y);
            int nN = y * nx + x;
            if (st->solid[nN]) continue;
            int nN1 = (y - oy) * nx + (x - ox);
            if (ox != 0) u[nN] = st->chi * u[nN1];
            else u[N + nN] = st->chi * u[N + nN1];
        }
    }

    /* 7. collision (Eq. 1) */
#pragma omp parallel for schedule(static) num_threads(nth)
    for (int n = 0; n < N; ++n) {
        if (st->solid[n]) {
            for (int k = 0; k < NCOMP; ++k)
                for (int i = 0; i < NQ; ++i) f[FIDX(k, i, n)] = 0.0;
            continue;
        }
        for (int k = 0; k < NCOMP; ++k) {
            double fin[NQ], fout[NQ];
            for (int i = 0; i < NQ; ++i) fin[i] = fp[FIDX(k, i, n)];
            orc_collide(fin, rho[(size_t)k * N + n], u[n], u[N + n],
                        F[((size_t)k * 2 + 0) * N + n], F[((size_t)k * 2 + 1) * N + n],
                        st->s[k], fout);
            for (int i = 0; i < NQ; ++i) f[FIDX(k, i, n)] = fout[i];
        }
    }

    /* 8. reductions that set lambda (Eq. 21) and chi (Eq. 23) for the next step */
    double qin, qout, usum;
    int have_in, mcount;
    int have_out = face_fluxes(st, &qin, &qout, &usum, &mcount, &have_in);
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

void orc_step(orc_state* st, int nsteps) {
    for (int s = 0; s < nsteps; ++s) one_step(st);
}

/* Fields of the last step: rho_k (2N), u^eq (2N), F_k (4N), all optional. */
void orc_get_macros(const orc_state* st, double* rho, double* u, double* F) {
    size_t N = (size_t)st->N;
    if (rho) memcpy(rho, st->rho, sizeof(double) * 2 * N);
    if (u) memcpy(u, st->u, sizeof(double) * 2 * N);
    if (F) memcpy(F, st->F, sizeof(double) * 4 * N);
}

/* Post-collision populations f*, [2][9][N]. */
void orc_get_f(const orc_state* st, double* f) {
    memcpy(f, st->f, sizeof(double) * NCOMP * NQ * (size_t)st->N);
}

void orc_set_f(orc_state* st, const double* f) {
    memcpy(st->f, f, sizeof(double) * NCOMP * NQ * (size_t)st->N);
}

/* Overwrite the post-stream, post-boundary populations of the last step
 * (the f_i(x_N, t) that Eq. 20 reads in the next step), [2][9][N]. */
void orc_set_fpost(orc_state* st, const double* f) {
    memcpy(st->fpost, f, sizeof(double) * NCOMP * NQ * (size_t)st->N);
}

/* Overwrite lambda (Eq. 21) and chi (Eq. 23) that the next step uses. */
void orc_set_outlet_coeffs(orc_state* st, double lambda, double chi) {
    st->lambda = lambda;
    st->chi = chi;
}

/* Post-stream, post-boundary populations of the last step, [2][9][N]. */
void orc_get_fpost(const orc_state* st, double* f) {
    memcpy(f, st->fpost, sizeof(double) * NCOMP * NQ * (size_t)st->N);
}

/* Forces of the step before the last one (the lagged forces the last
 * step's inlet used), [2][2][N]. */
void orc_get_force_prev(const orc_state* st, double* F) {
    memcpy(F, st->Fprev, sizeof(double) * NCOMP * 2 * (size_t)st->N);
}

/* out: [lambda, chi, Qin, Qout, Umean, mass_1, mass_2, step, s(2x9)...] */
void orc_get_scalars(const orc_state* st, double* out) {
    double m[NCOMP] = {0.0, 0.0};
    size_t N = (size_t)st->N;
    for (int k = 0; k < NCOMP; ++k)
        for (size_t n = 0; n < N; ++n)
            if (!st->solid[n])
                for (int i = 0; i < NQ; ++i) m[k] += st->f[FIDX(k, i, n)];
    out[0] = st->lambda;
    out[1] = st->chi;
    out[2] = st->Qin;
    out[3] = st->Qout;
    out[4] = st->Umean;
    out[5] = m[0];
    out[6] = m[1];
    out[7] = (double)st->step;
    for (int k = 0; k < NCOMP; ++k)
        for (int r = 0; r < NQ; ++r) out[8 + k * NQ + r] = st->s[k][r];
}

/* Forces of Eqs. 10/11 for given psi fields on the state's geometry (no
 * state change): psi [2][N] in, F [2][2][N] out. */
void orc_eval_forces(const orc_state* st, const double* psi, double* F) {
    int nx = st->nx, ny = st->ny, N = st->N;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int n = y * nx + x;
            double gx[2] = {0, 0}, gy[2] = {0, 0}, ax = 0, ay = 0;
            if (!st->solid[n])
                for (int c = 0; c < 24; ++c) {
                    int m;
                    if (psi_site(st, x + ST_DX[c], y + ST_DY[c], &m)) {
                        ax += ST_W[c] * ST_DX[c];
                        ay += ST_W[c] * ST_DY[c];
                    } else
                        for (int k = 0; k < 2; ++k) {
                            gx[k] += ST_W[c] * psi[(size_t)k * N + m] * ST_DX[c];
                            gy[k] += ST_W[c] * psi[(size_t)k * N + m] * ST_DY[c];
                        }
                }
            for (int k = 0; k < 2; ++k) {
                double pk = st->solid[n] ? 0.0 : psi[(size_t)k * N + n];
                const double gw = st->solid[n] ? 0.0 : adhesion_coeff(st, k, psi[n], psi[N + n]);
                F[((size_t)k * 2 + 0) * N + n] = -st->p.G12 * pk * gx[1 - k] - gw * pk * ax;
                F[((size_t)k * 2 + 1) * N + n] = -st->p.G12 * pk * gy[1 - k] - gw * pk * ay;
            }
        }
}
