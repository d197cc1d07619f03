/*
 * fdtd_oracle.c -- plain FP64 CPU FDTD used to check the CUDA library.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may load or call
 * this file: only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference legs of bench.py do.  It shares no code, header, table or
 * helper with the CUDA library; the two meet only through the seeded input
 * generators and the cell-owned field interchange layout described below.
 *
 * What it computes (Kuklin, "elecode", arXiv 2207.06908):
 *   - Sec. 2.1, Eq. (maxwell), (maxwelle), (maxwellh): lossy Maxwell curl
 *     equations with per-cell eps, sigma, mu.
 *   - Sec. 2.1, Eq. (fdtdex), (fdtdhx): Yee staggered updates of E and H.
 *     The loss term is taken in the semi-implicit (time-averaged sigma*E)
 *     form of the textbook the paper cites; Eq. (fdtdex) prints the explicit
 *     factor (1 - sigma dt / eps), which is unstable once sigma dt / eps > 2.
 *   - Sec. 2.1 (sources): ideal lumped current source on one Yee edge,
 *     J = I / dx^2 along +axis, I sampled at t_{n+1/2}; non-ideal current
 *     source (internal resistance R in parallel: an extra conductance
 *     1 / (R dx) on the edge, so the edge current is I + E dx / R);
 *     voltage sources (V = -E dx across the edge): ideal ones force
 *     E^{n+1} = -V(t_{n+1}) / dx, ones with internal resistance R in series
 *     act through their Norton equivalent, a current V(t_{n+1/2}) / R in
 *     parallel with R; lumped resistors and capacitors on one edge (current
 *     E dx / R and C dx dE/dt: an extra conductivity 1 / (R dx) and
 *     permittivity C / dx on that edge), the lumped-element forms of the
 *     textbook the paper cites.
 *   - Sec. 2.2: CPML absorbing layer (CFS recursive convolution, Roden and
 *     Gedney) terminated by PEC.
 *   - Sec. 2.3: thin wire by modified material parameters around a
 *     zero-tangential-E line: the radial E at the wire nodes get eps and
 *     sigma times m, every H those E read (circumferential and axial) gets
 *     mu / m, m = ln(dx / r0) / ln(dx / a), r0 = 0.23 dx, a <= r0.  The
 *     paper gives only references for the formula; the H set is widened
 *     beyond the circumferential H for stability (see orc_finalize).
 *   - Sec. 4 model files ("calculate"): voltage = -sum E dl along a path,
 *     current = loop integral of H around an edge.
 *   - Dispersive media (the paper's "Dispersive media" subsection): a
 *     multi-term Debye permittivity eps(w) = eps_inf + sum_p deps_p /
 *     (1 + j w tau_p) plus static sigma, by the auxiliary differential
 *     equation method of the references it cites (Okoniewski et al.;
 *     Taflove and Hagness): per pole a polarisation current J_p kept at the
 *     E time levels t_n, with tau_p dJ_p/dt + J_p = eps0 deps_p dE/dt taken
 *     by the trapezoidal rule over [t_n, t_{n+1}]; Ampere's law at
 *     t_{n+1/2} uses the mean of J_p^n and J_p^{n+1}.  Readings (the
 *     paper is silent): an E edge takes the mean over its four cells of each
 *     pole's deps (zero for cells without that pole) and the deps-weighted
 *     mean of its tau; a thin wire scales the whole complex permittivity
 *     (eps_inf, sigma and every deps_p) by its factor m.  The interface
 *     averaging of poles is parity unpinned against the paper.
 *   - Sec. 2.3 (oblique wires, the Guiffaut formalism the paper cites;
 *     the paper prints none of its equations, so this is a reading in the
 *     Holland-Simpson family it belongs to): a straight wire between two
 *     arbitrary points in node units, split into segments of about one
 *     cell; currents I_s at segment centres (times n+1/2) and charges Q_m
 *     at the wire nodes (times n).  Per unit length the wire carries the
 *     in-cell inductance L' = mu/(2 pi) ln(R/a), capacitance C' = 2 pi
 *     eps / ln(R/a) and leakage G' = 2 pi sigma / ln(R/a) between its
 *     radius a and the radius R at which the grid itself sees a line
 *     current: R = dx r0 exp(2 pi S), r0 = exp(-gamma) / (2 sqrt 2) (the
 *     square-lattice Green's function, G(0) - G(r) -> (ln(r/r0))/(2 pi)),
 *     S = sum over pairs i != j of w_i w_j (G(0) - G(r_ij)) for the
 *     bilinear weights w of the segment centre across the line lattice of
 *     its dominant axis (G(0) - G = 1/4 at one spacing, 1/pi on the
 *     diagonal).  Steps: I_s += dt/L' [E_s - (V_b - V_a)/dl], V_m = Q_m /
 *     (C' dl_m); the segment current enters Ampere's law at t_{n+1/2} as
 *     edge currents I W_e / dx^2 and E_s = sum_e W_e E_e^n dx / dl is the
 *     mean tangential E^n along it, with the same edge shares W_e both
 *     ways (reciprocal exchange).  W_e follow the charge-conserving
 *     deposition of particle codes (Villasenor and Buneman): the straight
 *     path a -> b is cut at the cell faces and each piece spreads its
 *     displacement over the 12 edges of its cell so that the grid's
 *     discrete divergence equals the move of a unit charge between the
 *     trilinear node weights of a and b; without it a steady current along
 *     an oblique wire would pile up spurious grid charge; Q_m^{n+1} = Q_m^n + dt [sum of currents into m] -
 *     (G'/C') dt (Q^{n+1} + Q^n)/2.  A source is a delta-gap EMF V(t_n) in
 *     one segment with a series resistance R: L' dl dI/dt = E_s dl - (V_b -
 *     V_a) + V - R I, the R I term at the mean of I^{n-1/2} and I^{n+1/2}
 *     (stable for any R).  Inside the CPML the wire is a matched lossy
 *     line, R'/L' = G'/C' = nu = sum_u t_u^2 sigma_u / (kappa_u eps0) (the
 *     layer's attenuation of a wave running along the wire; equal ratios
 *     keep its impedance), so its own wave is absorbed with the grid's;
 *     this is a reading, the paper is silent on wires in the layer; its
 *     t_u^2 weighting is pinned by isotropy: in a layer stretched alike
 *     along two axes a wire's wave decays alike in every direction of
 *     their plane (tests/test_owire_pins.py), which |t_u| would break.  In a
 *     Debye medium the in-cell capacitance takes the medium's dispersion
 *     (the Debye extension of thin wires the paper cites, in this form):
 *     K Q = eps0 eps_inf V + sum_p P_p with K = ln(R/a) / (2 pi dl_m),
 *     tau_p dP_p/dt + P_p = eps0 deps_p V, dQ/dt = (net current in) -
 *     (sigma / K) V, the last two by the trapezoidal rule; without poles
 *     this is the charge update above.  Wires
 *     whose end points coincide share that node (junction, Kirchhoff's
 *     current law); a node on an outer wall is grounded (V = 0), and so
 *     is a node on the node line of an axis-aligned wire: it joins that
 *     conductor, its charge handed to the grid (the PEC line carries it).
 *     The
 *     in-cell radius is parity unpinned against the paper (pinned by
 *     transmission-line impedance and rotation tests).
 *
 * Layout.  Every component is a node-indexed FP64 array of
 * (nx+1)(ny+1)(nz+1) entries, index (k*(ny+1)+j)*(nx+1)+i, holding
 *   Ex(i+1/2,j,k) Ey(i,j+1/2,k) Ez(i,j,k+1/2)
 *   Hx(i,j+1/2,k+1/2) Hy(i+1/2,j,k+1/2) Hz(i+1/2,j+1/2,k).
 * Entries at index nx, ny or nz along an axis are on the far walls and stay
 * zero.  Fields are exchanged with callers in the cell-owned layout: an
 * nx*ny*nz array, x fastest, entry (i,j,k) = the component with those
 * indices.
 *
 * Parity mode rounds every coefficient (ca, cb, db, the source factor, the
 * CPML b, c, 1/kappa) and every source sample to FP32 before use, so a
 * comparison with an FP32 GPU run measures arithmetic error only.  All
 * arithmetic stays FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Storage and update precision.  The oracle is FP64; the same source built
 * with -DORC_REAL=float gives a plain FP32 evaluation of the identical
 * algorithm, used only to size the rounding error FP32 storage cannot
 * avoid (never as a reference). */
#ifndef ORC_REAL
#define ORC_REAL double
#endif
typedef ORC_REAL real;

#define ORC_C0 299792458.0
#define ORC_EPS0 8.8541878128e-12
#define ORC_MU0 1.25663706212e-6
#define ORC_R0_FRAC 0.23
#define ORC_MAXP 4                 /* Debye poles per material */

enum { EX = 0, EY, EZ, HX, HY, HZ };
enum { PROBE_V = 0, PROBE_I = 1, PROBE_E = 2, PROBE_H = 3, PROBE_W = 4, PROBE_WV = 5 };

typedef struct { int axis, i, j, k, n; double radius; } orc_wire;
typedef struct { int axis, i, j, k, n; real *cur; int hard; } orc_src;   /* hard: ideal voltage source */
typedef struct { int axis, i, j, k; double e_add, s_add; } orc_lump;      /* extra eps (F/m), sigma (S/m) */
typedef struct { int kind, axis, i, j, k, n_edges; } orc_probe;

/* oblique wires: segments with their coupling edges, nodes, node sources */
#define ORC_OW_EDGES 48            /* up to 4 cells x 12 edges */
typedef struct {
    int a, b;                      /* wire nodes at the ends; I flows a -> b */
    double c[3], t[3], dl;         /* centre (node units), direction, length (m) */
    double lam;                    /* ln(R / a) */
    real cI;                       /* dt / L' */
    double R;                      /* series resistance of its sources (ohm) */
    double nu;                     /* CPML loss rate along it (1/s) */
    real rk, rd;                   /* (1 - k) / (1 + k), 1 / (1 + k), k = dt (R / (L' dl) + nu) / 2 */
    int ne;                        /* coupling edges */
    int comp[ORC_OW_EDGES];
    size_t q[ORC_OW_EDGES];
    double W[ORC_OW_EDGES];        /* edge share of the path (cell units, signed) */
    real wg[ORC_OW_EDGES];         /* gather: W dx / dl (E_s = sum wg E) */
    real ws[ORC_OW_EDGES];         /* scatter: cb_edge W / dx (E -= ws I) */
} orc_oseg;
typedef struct {
    double p[3];                   /* node units */
    double dlm, lam_sum, nu_sum;   /* wire length it carries (m); sums of ln(R/a) and CPML rate of its segments */
    int nadj, grounded;
    /* in-cell medium: K Q = e0 V + sum_p P_p (K = ln(R/a) / (2 pi dl_m));
     * Q^{n+1} = Q^n + dt (net current in) - (cs / K)(V^{n+1} + V^n);
     * P_p^{n+1} = pa_p P_p^n + pb_p (V^{n+1} + V^n) */
    real K, e0, cs, pa[ORC_MAXP], pb[ORC_MAXP];
    double cV;                     /* K / e0 (V per unit charge without poles) */
} orc_onode;
typedef struct { int seg0, nseg; double radius; } orc_owire;
typedef struct { int seg, n; real *emf; double r; } orc_osrc;   /* delta-gap EMF with series resistance r */

typedef struct orc_grid {
    int nx, ny, nz;
    double dx, dt, courant;
    int parity;
    size_t sy, sz, ntot;       /* strides of the node-indexed arrays */
    real *f[6];                /* Ex Ey Ez Hx Hy Hz */
    /* materials per cell */
    uint8_t *mat;
    double *m_eps, *m_sig, *m_mu;
    int n_mat;
    /* coefficients per component position */
    real *ca[3], *cb[3], *db[3];
    /* CPML */
    int d;
    double order, kappa_max, alpha_max, alpha_order, sigma_max;
    /* profile per axis u: E-position (integer node) and H-position
     * (half-integer) b, c, 1/kappa, plus an "inside the layer" flag */
    real *pe_b[3], *pe_c[3], *pe_ki[3];
    real *ph_b[3], *ph_c[3], *ph_ki[3];
    uint8_t *pe_on[3], *ph_on[3];
    /* psi[comp][axis]: auxiliary field of component comp (0..5) for its
     * derivative along axis; full node-indexed arrays, NULL on the diagonal */
    real *psi[6][3];
    /* wires, sources, probes */
    orc_wire *wires; int n_wires;
    orc_src *srcs; int n_srcs;
    orc_lump *lumps; int n_lumps;
    real *hard_coef;           /* -1/dx per hard source (0 for current sources) */
    orc_probe *probes; int n_probes;
    real *src_coef;            /* -cb/dx at each source edge */
    /* Debye media: poles per material (deps_p, tau_p; deps 0 = no pole);
     * per E edge and pole: cj (E^{n+1} += cj J^n), k and be (J^{n+1} =
     * k J^n + be (E^{n+1} - E^n)) and the current J_p^n (at the E time
     * level); allocated when any material has a pole */
    double m_deps[256][ORC_MAXP], m_tau[256][ORC_MAXP];
    int has_debye;
    real *dcj[3][ORC_MAXP], *dk[3][ORC_MAXP], *dbe[3][ORC_MAXP], *J[3][ORC_MAXP];
    real *eprev[3];
    /* oblique wires: segments, nodes, wires, node current sources and the
     * state I_s^{n-1/2} (before a step), Q_m^n */
    orc_oseg *osegs; int n_osegs;
    orc_onode *onodes; int n_onodes;
    orc_owire *owires; int n_owires;
    orc_osrc *osrcs; int n_osrcs;
    double *oI, *oQ, *oV, *oP;     /* oP: [node][ORC_MAXP] */
    int max_steps;
    double *probe_out;         /* [n_probes][max_steps] */
    long step;
    int finalized;
} orc_grid;

static double r32(const orc_grid *g, double v) { return g->parity ? (double)(float)v : v; }

static inline size_t IDX(const orc_grid *g, int i, int j, int k)
{
    return ((size_t)k * g->sz) + ((size_t)j * g->sy) + (size_t)i;
}

static inline int CELL(const orc_grid *g, int i, int j, int k)
{
    return (k * g->ny + j) * g->nx + i;
}

orc_grid *orc_create(int nx, int ny, int nz, double dx, double courant, int parity)
{
    if (nx < 2 || ny < 2 || nz < 2 || !(dx > 0) || !(courant > 0)) return NULL;
    orc_grid *g = (orc_grid *)calloc(1, sizeof(orc_grid));
    g->nx = nx; g->ny = ny; g->nz = nz; g->dx = dx; g->courant = courant;
    /* Courant limit for a uniform cubic grid: c dt <= dx / sqrt(3) */
    g->dt = courant * dx / (ORC_C0 * sqrt(3.0));
    g->parity = parity;
    g->sy = (size_t)(nx + 1);
    g->sz = (size_t)(nx + 1) * (size_t)(ny + 1);
    g->ntot = g->sz * (size_t)(nz + 1);
    for (int c = 0; c < 6; c++) g->f[c] = (real *)calloc(g->ntot, sizeof(real));
    g->mat = (uint8_t *)calloc((size_t)nx * ny * nz, 1);
    g->n_mat = 1;
    g->m_eps = (double *)malloc(sizeof(double)); g->m_eps[0] = 1.0;
    g->m_sig = (double *)malloc(sizeof(double)); g->m_sig[0] = 0.0;
    g->m_mu = (double *)malloc(sizeof(double)); g->m_mu[0] = 1.0;
    return g;
}

void orc_destroy(orc_grid *g)
{
    if (!g) return;
    for (int c = 0; c < 6; c++) free(g->f[c]);
    for (int c = 0; c < 3; c++) { free(g->ca[c]); free(g->cb[c]); free(g->db[c]); }
    for (int u = 0; u < 3; u++) {
        free(g->pe_b[u]); free(g->pe_c[u]); free(g->pe_ki[u]); free(g->pe_on[u]);
        free(g->ph_b[u]); free(g->ph_c[u]); free(g->ph_ki[u]); free(g->ph_on[u]);
    }
    for (int c = 0; c < 6; c++) for (int u = 0; u < 3; u++) free(g->psi[c][u]);
    for (int c = 0; c < 3; c++) {
        free(g->eprev[c]);
        for (int p = 0; p < ORC_MAXP; p++) { free(g->dcj[c][p]); free(g->dk[c][p]); free(g->dbe[c][p]); free(g->J[c][p]); }
    }
    for (int s = 0; s < g->n_srcs; s++) free(g->srcs[s].cur);
    free(g->srcs); free(g->wires); free(g->probes); free(g->src_coef); free(g->probe_out);
    free(g->lumps); free(g->hard_coef);
    for (int s = 0; s < g->n_osrcs; s++) free(g->osrcs[s].emf);
    free(g->osegs); free(g->onodes); free(g->owires); free(g->osrcs); free(g->oI); free(g->oQ);
    free(g->oV); free(g->oP);
    free(g->mat); free(g->m_eps); free(g->m_sig); free(g->m_mu);
    free(g);
}

double orc_dt(const orc_grid *g) { return g->dt; }

/* number of OpenMP threads the update loops use */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
long orc_step_count(const orc_grid *g) { return g->step; }

/* sigma_max <= 0 selects 0.8 (m+1) / (eta0 dx), the usual optimum for a
 * polynomial grading of order m. */
int orc_set_cpml(orc_grid *g, int d, double order, double kappa_max, double alpha_max,
                 double alpha_order, double sigma_max)
{
    if (g->finalized) return -8;
    if (d < 0 || 2 * d > g->nx || 2 * d > g->ny || 2 * d > g->nz) return -1;
    g->d = d; g->order = order; g->kappa_max = kappa_max; g->alpha_max = alpha_max;
    g->alpha_order = alpha_order;
    if (sigma_max <= 0) {
        double eta0 = sqrt(ORC_MU0 / ORC_EPS0);
        sigma_max = 0.8 * (order + 1.0) / (eta0 * g->dx);
    }
    g->sigma_max = sigma_max;
    return 0;
}

int orc_set_materials(orc_grid *g, const uint8_t *cell_mat, const double *eps_r,
                      const double *sigma, const double *mu_r, int n_mat)
{
    if (g->finalized) return -8;
    if (n_mat < 1 || n_mat > 256) return -1;
    size_t nc = (size_t)g->nx * g->ny * g->nz;
    for (size_t c = 0; c < nc; c++) if (cell_mat[c] >= n_mat) return -1;
    memcpy(g->mat, cell_mat, nc);
    free(g->m_eps); free(g->m_sig); free(g->m_mu);
    g->m_eps = (double *)malloc(n_mat * sizeof(double));
    g->m_sig = (double *)malloc(n_mat * sizeof(double));
    g->m_mu = (double *)malloc(n_mat * sizeof(double));
    memcpy(g->m_eps, eps_r, n_mat * sizeof(double));
    memcpy(g->m_sig, sigma, n_mat * sizeof(double));
    memcpy(g->m_mu, mu_r, n_mat * sizeof(double));
    g->n_mat = n_mat;
    return 0;
}

/* Wire between two arbitrary nodes as a staircase of grid-aligned
 * segments (the staircase wire model the paper lists among its thin-wire
 * techniques): from a, each unit step goes along the axis whose progress
 * towards b, |c_u - a_u| / |b_u - a_u|, is smallest (ties: lowest axis);
 * runs of steps along one axis form one wire.  Returns the number of
 * wires added, or a negative status. */
int orc_add_wire(orc_grid *g, int i0, int j0, int k0, int i1, int j1, int k1, double radius);

int orc_add_wire_path(orc_grid *g, int i0, int j0, int k0, int i1, int j1, int k1, double radius)
{
    if (g->finalized) return -8;
    int a[3] = {i0, j0, k0}, b[3] = {i1, j1, k1}, c[3] = {i0, j0, k0};
    int d[3], len = 0;
    for (int u = 0; u < 3; u++) { d[u] = abs(b[u] - a[u]); len += d[u]; }
    if (len == 0) return -1;
    int run_axis = -1, run_start[3] = {0, 0, 0}, added = 0;
    for (int s = 0; s <= len; s++) {
        int best = -1;
        if (s < len) {
            double bp = 2.0;
            for (int u = 0; u < 3; u++) {
                if (c[u] == b[u]) continue;
                double prog = (double)abs(c[u] - a[u]) / d[u];
                if (prog < bp) { bp = prog; best = u; }
            }
        }
        if (best != run_axis) {
            if (run_axis >= 0) {            /* close the run from run_start to c */
                int p0[3] = {run_start[0], run_start[1], run_start[2]}, p1[3] = {c[0], c[1], c[2]};
                if (p1[run_axis] < p0[run_axis]) { int t = p0[run_axis]; p0[run_axis] = p1[run_axis]; p1[run_axis] = t; }
                int rc = orc_add_wire(g, p0[0], p0[1], p0[2], p1[0], p1[1], p1[2], radius);
                if (rc) return rc;
                added++;
            }
            run_axis = best;
            for (int u = 0; u < 3; u++) run_start[u] = c[u];
        }
        if (best >= 0) c[best] += b[best] > a[best] ? 1 : -1;
    }
    return added;
}

/* Debye poles of material `mat`: deps[p] (relative, >= 0) and tau[p] (s,
 * > 0), p < n_poles <= ORC_MAXP; later poles are cleared */
int orc_set_debye(orc_grid *g, int mat, int n_poles, const double *deps, const double *tau)
{
    if (g->finalized) return -8;
    if (mat < 0 || mat > 255 || n_poles < 0 || n_poles > ORC_MAXP) return -1;
    for (int p = 0; p < n_poles; p++)
        if (!(deps[p] >= 0) || !(tau[p] > 0)) return -1;
    for (int p = 0; p < ORC_MAXP; p++) {
        g->m_deps[mat][p] = p < n_poles ? deps[p] : 0.0;
        g->m_tau[mat][p] = p < n_poles ? tau[p] : 1.0;
        if (g->m_deps[mat][p] > 0) g->has_debye = 1;
    }
    return 0;
}

/* axis-aligned wire from node (i0,j0,k0) to node (i1,j1,k1) */
int orc_add_wire(orc_grid *g, int i0, int j0, int k0, int i1, int j1, int k1, double radius)
{
    if (g->finalized) return -8;
    int axis, n;
    if (j0 == j1 && k0 == k1 && i1 > i0) { axis = 0; n = i1 - i0; }
    else if (i0 == i1 && k0 == k1 && j1 > j0) { axis = 1; n = j1 - j0; }
    else if (i0 == i1 && j0 == j1 && k1 > k0) { axis = 2; n = k1 - k0; }
    else return -1;
    /* m <= 1 (a <= r0): thicker wires would need the opposite stability rule */
    if (!(radius > 0) || radius > ORC_R0_FRAC * g->dx * (1.0 + 1e-12)) return -1;
    /* the wire and its neighbouring radial/circumferential components must
     * lie strictly inside the walls */
    int lo[3] = {i0, j0, k0}, hi[3] = {i1, j1, k1}, nn[3] = {g->nx, g->ny, g->nz};
    for (int u = 0; u < 3; u++) {
        if (u == axis) { if (lo[u] < 0 || hi[u] > nn[u]) return -1; }
        else if (lo[u] < 1 || lo[u] > nn[u] - 1) return -1;
    }
    g->wires = (orc_wire *)realloc(g->wires, (g->n_wires + 1) * sizeof(orc_wire));
    orc_wire w = {axis, i0, j0, k0, n, radius};
    g->wires[g->n_wires++] = w;
    return 0;
}

static int edge_ok(const orc_grid *g, int i, int j, int k, int axis)
{
    if (axis < 0 || axis > 2) return 0;
    int p[3] = {i, j, k}, nn[3] = {g->nx, g->ny, g->nz};
    for (int u = 0; u < 3; u++) {
        if (u == axis) { if (p[u] < 0 || p[u] >= nn[u]) return 0; }
        else if (p[u] < 1 || p[u] > nn[u] - 1) return 0;
    }
    return 1;
}

static int add_lump(orc_grid *g, int i, int j, int k, int axis, double e_add, double s_add)
{
    g->lumps = (orc_lump *)realloc(g->lumps, (g->n_lumps + 1) * sizeof(orc_lump));
    orc_lump l = {axis, i, j, k, e_add, s_add};
    g->lumps[g->n_lumps++] = l;
    return 0;
}

static int push_src(orc_grid *g, int i, int j, int k, int axis, const double *v, int n, double scale, int hard)
{
    g->srcs = (orc_src *)realloc(g->srcs, (g->n_srcs + 1) * sizeof(orc_src));
    orc_src s = {axis, i, j, k, n, NULL, hard};
    s.cur = (real *)malloc((n > 0 ? n : 1) * sizeof(real));
    for (int t = 0; t < n; t++) s.cur[t] = r32(g, v[t] * scale);
    g->srcs[g->n_srcs++] = s;
    return 0;
}

/* current source on the edge from node (i,j,k) along +axis; r_internal > 0:
 * in parallel with that resistance (ohm) */
int orc_add_source_r(orc_grid *g, int i, int j, int k, int axis, double r_internal, const double *cur, int n)
{
    if (g->finalized) return -8;
    if (n < 0 || !edge_ok(g, i, j, k, axis) || !(r_internal >= 0)) return -1;
    if (r_internal > 0) add_lump(g, i, j, k, axis, 0.0, 1.0 / (r_internal * g->dx));
    return push_src(g, i, j, k, axis, cur, n, 1.0, 0);
}

int orc_add_source(orc_grid *g, int i, int j, int k, int axis, const double *cur, int n)
{
    return orc_add_source_r(g, i, j, k, axis, 0.0, cur, n);
}

/* voltage source across the edge (V = -E dx): r_internal = 0 ideal (volt[n]
 * is V at t_{n+1}), > 0 in series with that resistance (volt[n] at
 * t_{n+1/2}, applied as the current volt / r in parallel with r) */
int orc_add_vsource(orc_grid *g, int i, int j, int k, int axis, double r_internal, const double *volt, int n)
{
    if (g->finalized) return -8;
    if (n < 0 || !edge_ok(g, i, j, k, axis) || !(r_internal >= 0)) return -1;
    if (r_internal == 0) return push_src(g, i, j, k, axis, volt, n, 1.0, 1);
    add_lump(g, i, j, k, axis, 0.0, 1.0 / (r_internal * g->dx));
    return push_src(g, i, j, k, axis, volt, n, 1.0 / r_internal, 0);
}

/* lumped resistor (ohm, 0 = none) and / or capacitor (F, 0 = none) on the
 * edge from node (i,j,k) along +axis */
int orc_add_lumped(orc_grid *g, int i, int j, int k, int axis, double resistance, double capacitance)
{
    if (g->finalized) return -8;
    if (!edge_ok(g, i, j, k, axis) || !(resistance >= 0) || !(capacitance >= 0)) return -1;
    return add_lump(g, i, j, k, axis, capacitance / g->dx, resistance > 0 ? 1.0 / (resistance * g->dx) : 0.0);
}

int orc_add_probe(orc_grid *g, int kind, int i, int j, int k, int axis, int n_edges)
{
    if (g->finalized) return -8;
    if (kind >= PROBE_W) return -1;    /* oblique-wire probes have their own calls */
    if (axis < 0 || axis > 2 || kind < 0 || kind > 3) return -1;
    int p[3] = {i, j, k}, nn[3] = {g->nx, g->ny, g->nz};
    for (int u = 0; u < 3; u++) if (p[u] < 0 || p[u] >= nn[u]) return -1;
    if (kind == PROBE_V) { if (n_edges < 1 || p[axis] + n_edges > nn[axis]) return -1; }
    else n_edges = 1;
    if (kind == PROBE_I) {
        for (int u = 0; u < 3; u++) if (u != axis && p[u] < 1) return -1;
    }
    g->probes = (orc_probe *)realloc(g->probes, (g->n_probes + 1) * sizeof(orc_probe));
    orc_probe pr = {kind, axis, i, j, k, n_edges};
    g->probes[g->n_probes++] = pr;
    return 0;
}

/* material of cell (i,j,k); cells outside the grid are never asked for */
static double cell_eps(const orc_grid *g, int i, int j, int k) { return g->m_eps[g->mat[CELL(g, i, j, k)]]; }
static double cell_sig(const orc_grid *g, int i, int j, int k) { return g->m_sig[g->mat[CELL(g, i, j, k)]]; }
static double cell_mu(const orc_grid *g, int i, int j, int k) { return g->m_mu[g->mat[CELL(g, i, j, k)]]; }

/* ---- oblique wires --------------------------------------------------------
 * A straight wire from (x0,y0,z0) to (x1,y1,z1) in node units (point (i,j,k)
 * is at (i dx, j dx, k dx)), radius in metres, split into round(length in
 * cells) segments (at least one).  End points that coincide with a node of
 * an earlier oblique wire join it (junction).  Returns the wire index. */
static int onode_at(const orc_grid *g, const double p[3])
{
    for (int m = 0; m < g->n_onodes; m++)
        if (fabs(g->onodes[m].p[0] - p[0]) < 1e-9 && fabs(g->onodes[m].p[1] - p[1]) < 1e-9 &&
            fabs(g->onodes[m].p[2] - p[2]) < 1e-9)
            return m;
    return -1;
}

static int onode_new(orc_grid *g, const double p[3])
{
    g->onodes = (orc_onode *)realloc(g->onodes, (g->n_onodes + 1) * sizeof(orc_onode));
    orc_onode nd;
    memset(&nd, 0, sizeof nd);
    int nn[3] = {g->nx, g->ny, g->nz};
    for (int u = 0; u < 3; u++) {
        nd.p[u] = p[u];
        if (p[u] == 0.0 || p[u] == (double)nn[u]) nd.grounded = 1;
    }
    g->onodes[g->n_onodes] = nd;
    return g->n_onodes++;
}

int orc_add_owire(orc_grid *g, double x0, double y0, double z0, double x1, double y1, double z1, double radius)
{
    if (g->finalized) return -8;
    double A[3] = {x0, y0, z0}, B[3] = {x1, y1, z1};
    int nn[3] = {g->nx, g->ny, g->nz};
    double len = 0.0;
    for (int u = 0; u < 3; u++) {
        if (!(A[u] >= 0.0 && A[u] <= nn[u] && B[u] >= 0.0 && B[u] <= nn[u])) return -1;
        len += (B[u] - A[u]) * (B[u] - A[u]);
    }
    len = sqrt(len);
    if (!(len >= 0.5) || !(radius > 0.0) || radius > 0.1 * g->dx) return -1;
    int N = (int)lround(len);
    if (N < 1) N = 1;
    g->owires = (orc_owire *)realloc(g->owires, (g->n_owires + 1) * sizeof(orc_owire));
    orc_owire w = {g->n_osegs, N, radius};
    g->owires[g->n_owires] = w;
    int prev = onode_at(g, A);
    if (prev < 0) prev = onode_new(g, A);
    for (int sg = 0; sg < N; sg++) {
        double P[3];
        for (int u = 0; u < 3; u++) P[u] = A[u] + (B[u] - A[u]) * (double)(sg + 1) / N;
        int next = -1;
        if (sg == N - 1) { for (int u = 0; u < 3; u++) P[u] = B[u]; next = onode_at(g, B); }
        if (next < 0) next = onode_new(g, P);
        g->osegs = (orc_oseg *)realloc(g->osegs, (g->n_osegs + 1) * sizeof(orc_oseg));
        orc_oseg *S = &g->osegs[g->n_osegs++];
        memset(S, 0, sizeof *S);
        S->a = prev;
        S->b = next;
        for (int u = 0; u < 3; u++) {
            S->t[u] = (B[u] - A[u]) / len;
            S->c[u] = A[u] + (B[u] - A[u]) * (sg + 0.5) / N;
        }
        S->dl = len * g->dx / N;
        prev = next;
    }
    return g->n_owires++;
}

/* delta-gap EMF in segment seg of oblique wire w with series resistance r
 * (ohm, >= 0): volt[n] (V at t_n) drives the segment's current from its start
 * node to its end node */
int orc_add_owire_vsource(orc_grid *g, int w, int seg, double r, const double *volt, int n)
{
    if (g->finalized) return -8;
    if (w < 0 || w >= g->n_owires || seg < 0 || seg >= g->owires[w].nseg || n < 0 || !(r >= 0.0)) return -1;
    g->osrcs = (orc_osrc *)realloc(g->osrcs, (g->n_osrcs + 1) * sizeof(orc_osrc));
    orc_osrc sr = {g->owires[w].seg0 + seg, n, (real *)malloc((n > 0 ? n : 1) * sizeof(real)), r};
    for (int q = 0; q < n; q++) sr.emf[q] = r32(g, volt[q]);
    g->osrcs[g->n_osrcs++] = sr;
    return 0;
}

/* probe of segment seg of oblique wire w: I_s at t_{n+1/2} */
int orc_add_owire_probe(orc_grid *g, int w, int seg)
{
    if (g->finalized) return -8;
    if (w < 0 || w >= g->n_owires || seg < 0 || seg >= g->owires[w].nseg) return -1;
    g->probes = (orc_probe *)realloc(g->probes, (g->n_probes + 1) * sizeof(orc_probe));
    orc_probe pr = {PROBE_W, 0, g->owires[w].seg0 + seg, 0, 0, 1};
    g->probes[g->n_probes++] = pr;
    return 0;
}

/* probe of the in-cell potential Q_m / (C' dl_m) of the oblique-wire node at
 * (x, y, z) (node units), at t_{n+1}: added to a grid voltage path that ends
 * at the node it gives the wire's own potential */
int orc_add_owire_node_probe(orc_grid *g, double x, double y, double z)
{
    if (g->finalized) return -8;
    double P[3] = {x, y, z};
    int m = onode_at(g, P);
    if (m < 0) return -1;
    g->probes = (orc_probe *)realloc(g->probes, (g->n_probes + 1) * sizeof(orc_probe));
    orc_probe pr = {PROBE_WV, 0, m, 0, 0, 1};
    g->probes[g->n_probes++] = pr;
    return 0;
}

void orc_owire_counts(const orc_grid *g, int *n_seg, int *n_node)
{
    *n_seg = g->n_osegs;
    *n_node = g->n_onodes;
}

/* state I_s (last half step) and Q_m (current integer step) */
int orc_get_owire_state(const orc_grid *g, double *I, double *Q)
{
    if (!g->finalized) return -8;
    for (int s = 0; s < g->n_osegs; s++) I[s] = g->oI[s];
    for (int m = 0; m < g->n_onodes; m++) Q[m] = g->oQ[m];
    return 0;
}

int orc_set_owire_state(orc_grid *g, const double *I, const double *Q)
{
    if (!g->finalized) return -8;
    for (int s = 0; s < g->n_osegs; s++) g->oI[s] = I[s];
    for (int m = 0; m < g->n_onodes; m++) {
        /* the charge with its medium polarisation-free: V = K Q / e0 */
        const orc_onode *nd = &g->onodes[m];
        g->oQ[m] = nd->grounded ? 0.0 : Q[m];
        g->oV[m] = nd->grounded ? 0.0 : (double)nd->K * g->oQ[m] / (double)nd->e0;
        for (int p = 0; p < ORC_MAXP; p++) g->oP[(size_t)m * ORC_MAXP + p] = 0.0;
    }
    return 0;
}

/* per segment L' dl (H) and per node 1 / (C' dl_m) (1/F; 0 when grounded),
 * the quantities of the wire's stored energy */
int orc_get_owire_coefs(const orc_grid *g, double *Ldl, double *cV)
{
    if (!g->finalized) return -8;
    for (int s = 0; s < g->n_osegs; s++) {
        const orc_oseg *S = &g->osegs[s];
        int ci[3], nn[3] = {g->nx, g->ny, g->nz};
        for (int u = 0; u < 3; u++) {
            ci[u] = (int)floor(S->c[u]);
            if (ci[u] > nn[u] - 1) ci[u] = nn[u] - 1;
        }
        Ldl[s] = ORC_MU0 * cell_mu(g, ci[0], ci[1], ci[2]) * S->lam / (2.0 * M_PI) * S->dl;
    }
    for (int m = 0; m < g->n_onodes; m++) cV[m] = g->onodes[m].grounded ? 0.0 : g->onodes[m].cV;
    return 0;
}

/* the four cells around E edge comp at node (i,j,k) (the same cells whose
 * eps and sigma are averaged) */
static void edge_cells(int comp, int i, int j, int k, int cell[4][3])
{
    for (int t = 0; t < 4; t++) {
        int a = t & 1, b = t >> 1;
        if (comp == 0) { cell[t][0] = i; cell[t][1] = j - 1 + a; cell[t][2] = k - 1 + b; }
        else if (comp == 1) { cell[t][0] = i - 1 + a; cell[t][1] = j; cell[t][2] = k - 1 + b; }
        else { cell[t][0] = i - 1 + a; cell[t][1] = j - 1 + b; cell[t][2] = k; }
    }
}

/* Debye poles of an E edge: deps = mean over its four cells, tau = the
 * deps-weighted mean over the cells that have the pole */
static void edge_poles(const orc_grid *g, int comp, int i, int j, int k, double deps[ORC_MAXP],
                       double tau[ORC_MAXP])
{
    int cell[4][3];
    edge_cells(comp, i, j, k, cell);
    for (int p = 0; p < ORC_MAXP; p++) {
        double sd = 0.0, st = 0.0;
        for (int t = 0; t < 4; t++) {
            int m = g->mat[CELL(g, cell[t][0], cell[t][1], cell[t][2])];
            sd += g->m_deps[m][p];
            st += g->m_deps[m][p] * g->m_tau[m][p];
        }
        deps[p] = 0.25 * sd;
        tau[p] = sd > 0 ? st / sd : 1.0;
    }
}

/* coefficients of one E edge: eps (relative, averaged), sigma, wire factor
 * m; poles (deps relative, tau) when the edge is dispersive.  Without poles
 * the semi-implicit loss form ca = (1-a)/(1+a), cb = dt/(eps dx)/(1+a),
 * a = sigma dt / (2 eps); with poles the ADE form
 *   D = 2 eps + sum beta_p + sigma dt,
 *   ca = (2 eps + sum beta_p - sigma dt) / D,  cb = 2 dt / (D dx),
 *   cj_p = -dt (1 + k_p) / D,  k_p = (2 tau_p - dt) / (2 tau_p + dt),
 *   be_p = beta_p / dt,  beta_p = 2 eps0 deps_p dt / (2 tau_p + dt),
 * with eps, sigma and every deps scaled by m, and e_add, s_add (lumped
 * capacitance / dx, conductance / dx) added after the scaling. */
static int e_coefs(const orc_grid *g, double eps_r, double sig, double m, double e_add, double s_add,
                   const double *deps, const double *tau, double *ca, double *cb, double cj[ORC_MAXP],
                   double kk[ORC_MAXP], double be[ORC_MAXP])
{
    double dt = g->dt, dx = g->dx;
    double e = ORC_EPS0 * eps_r * m + e_add, s = sig * m + s_add;
    int disp = 0;
    for (int p = 0; p < ORC_MAXP; p++) {
        cj[p] = kk[p] = be[p] = 0.0;
        if (deps && deps[p] > 0) disp = 1;
    }
    if (!disp) {
        double a = s * dt / (2.0 * e);
        *ca = (1.0 - a) / (1.0 + a);
        *cb = dt / (e * dx) / (1.0 + a);
        return 0;
    }
    double beta[ORC_MAXP], sb = 0.0;
    for (int p = 0; p < ORC_MAXP; p++) {
        beta[p] = 2.0 * ORC_EPS0 * deps[p] * m * dt / (2.0 * tau[p] + dt);
        kk[p] = deps[p] > 0 ? (2.0 * tau[p] - dt) / (2.0 * tau[p] + dt) : 0.0;
        sb += beta[p];
    }
    double D = 2.0 * e + sb + s * dt;
    *ca = (2.0 * e + sb - s * dt) / D;
    *cb = 2.0 * dt / (D * dx);
    for (int p = 0; p < ORC_MAXP; p++) {
        if (!(deps[p] > 0)) continue;
        cj[p] = -dt * (1.0 + kk[p]) / D;
        be[p] = beta[p] / dt;
    }
    return 1;
}

/* CPML grading at depth rho (cells) into the layer, Roden-Gedney CFS form */
static void cpml_coef(const orc_grid *g, double rho, double *b, double *c, double *ki)
{
    double x = rho / g->d;
    double sig = g->sigma_max * pow(x, g->order);
    double kap = 1.0 + (g->kappa_max - 1.0) * pow(x, g->order);
    double alp = g->alpha_max * pow(1.0 - x, g->alpha_order);
    double bb = exp(-(sig / kap + alp) * g->dt / ORC_EPS0);
    double cc = (sig > 0) ? sig * (bb - 1.0) / (sig * kap + kap * kap * alp) : 0.0;
    *b = bb; *c = cc; *ki = 1.0 / kap;
}

static void build_cpml(orc_grid *g)
{
    int nn[3] = {g->nx, g->ny, g->nz};
    for (int u = 0; u < 3; u++) {
        int n = nn[u];
        g->pe_b[u] = (real *)calloc(n + 1, sizeof(real));
        g->pe_c[u] = (real *)calloc(n + 1, sizeof(real));
        g->pe_ki[u] = (real *)calloc(n + 1, sizeof(real));
        g->pe_on[u] = (uint8_t *)calloc(n + 1, 1);
        g->ph_b[u] = (real *)calloc(n + 1, sizeof(real));
        g->ph_c[u] = (real *)calloc(n + 1, sizeof(real));
        g->ph_ki[u] = (real *)calloc(n + 1, sizeof(real));
        g->ph_on[u] = (uint8_t *)calloc(n + 1, 1);
        for (int i = 0; i <= n; i++) {
            g->pe_ki[u][i] = 1.0; g->ph_ki[u][i] = 1.0; g->pe_b[u][i] = 1.0; g->ph_b[u][i] = 1.0;
        }
        if (g->d == 0) continue;
        int d = g->d;
        /* integer node positions i: depth d - i on the low side, i - (n - d)
         * on the high side; the layer interior is depth > 0 */
        for (int i = 0; i <= n; i++) {
            double rho = 0.0;
            if (i < d) rho = d - i;
            else if (i > n - d) rho = i - (n - d);
            if (rho > 0) {
                double b, c, ki; cpml_coef(g, rho, &b, &c, &ki);
                g->pe_b[u][i] = r32(g, b); g->pe_c[u][i] = r32(g, c); g->pe_ki[u][i] = r32(g, ki);
                g->pe_on[u][i] = 1;
            }
        }
        /* half-integer positions i + 1/2, i = 0..n-1 */
        for (int i = 0; i < n; i++) {
            double rho = 0.0;
            if (i < d) rho = d - (i + 0.5);
            else if (i >= n - d) rho = (i + 0.5) - (n - d);
            if (rho > 0) {
                double b, c, ki; cpml_coef(g, rho, &b, &c, &ki);
                g->ph_b[u][i] = r32(g, b); g->ph_c[u][i] = r32(g, c); g->ph_ki[u][i] = r32(g, ki);
                g->ph_on[u][i] = 1;
            }
        }
    }
    if (g->d == 0) return;
    /* psi arrays: component c has derivatives along the two other axes */
    int comp_axis[6] = {0, 1, 2, 0, 1, 2};
    for (int c = 0; c < 6; c++)
        for (int u = 0; u < 3; u++)
            if (u != comp_axis[c]) g->psi[c][u] = (real *)calloc(g->ntot, sizeof(real));
}

/* equivalent-radius factor of a thin wire of radius a (Sec. 2.3 reading) */
static double wire_factor(const orc_grid *g, double a)
{
    return log(g->dx / (ORC_R0_FRAC * g->dx)) / log(g->dx / a);
}

/* true when E component comp at node-index q is updated (not on a wall) */
static int e_interior(const orc_grid *g, int comp, const int q[3])
{
    int nn[3] = {g->nx, g->ny, g->nz};
    for (int u = 0; u < 3; u++) {
        if (u == comp) { if (q[u] < 0 || q[u] >= nn[u]) return 0; }
        else if (q[u] < 1 || q[u] > nn[u] - 1) return 0;
    }
    return 1;
}

/* the four H entries read by the update of E component comp at q, in the
 * order of the update stencils of update_e():
 *   Ex(i+1/2,j,k): Hz[i][j][k], Hz[i][j-1][k], Hy[i][j][k], Hy[i][j][k-1]
 *   Ey(i,j+1/2,k): Hx[i][j][k], Hx[i][j][k-1], Hz[i][j][k], Hz[i-1][j][k]
 *   Ez(i,j,k+1/2): Hy[i][j][k], Hy[i-1][j][k], Hx[i][j][k], Hx[i][j-1][k] */
static void e_stencil(int comp, const int q[3], int hc[4], int hp[4][3])
{
    int b = (comp + 1) % 3, c = (comp + 2) % 3;
    /* E_comp reads H_c differenced along b and H_b differenced along c */
    hc[0] = c; hc[1] = c; hc[2] = b; hc[3] = b;     /* H axis 0..2 */
    for (int t = 0; t < 4; t++) { hp[t][0] = q[0]; hp[t][1] = q[1]; hp[t][2] = q[2]; }
    hp[1][b] -= 1;
    hp[3][c] -= 1;
}


/* CPML attenuation rate sigma/(kappa eps0) along axis u at position x (cells) */
static double cpml_rate(const orc_grid *g, int u, double x)
{
    if (g->d == 0) return 0.0;
    int nn[3] = {g->nx, g->ny, g->nz};
    double rho = 0.0;
    if (x < g->d) rho = g->d - x;
    else if (x > nn[u] - g->d) rho = x - (nn[u] - g->d);
    if (rho <= 0.0) return 0.0;
    double r = rho / g->d;
    double sig = g->sigma_max * pow(r, g->order), kap = 1.0 + (g->kappa_max - 1.0) * pow(r, g->order);
    return sig / (kap * ORC_EPS0);
}

/* in-cell parameters and coupling edges of the oblique wires (after the
 * E coefficients exist: the scatter uses each edge's cb) */
/* does point p (node units) lie on the node line of axis-aligned wire w */
static int on_axis_wire(const orc_wire *w, const double p[3])
{
    const int c[3] = {w->i, w->j, w->k};
    for (int u = 0; u < 3; u++) {
        if (u == w->axis) {
            if (p[u] < c[u] - 1e-9 || p[u] > c[u] + w->n + 1e-9) return 0;
        } else if (fabs(p[u] - c[u]) > 1e-9) {
            return 0;
        }
    }
    return 1;
}

static int build_owires(orc_grid *g)
{
    const double dx = g->dx, dt = g->dt;
    const double r0 = exp(-0.57721566490153286) / (2.0 * sqrt(2.0));
    int nn[3] = {g->nx, g->ny, g->nz};
    for (int m = 0; m < g->n_onodes; m++) {
        g->onodes[m].dlm = 0.0; g->onodes[m].lam_sum = 0.0; g->onodes[m].nu_sum = 0.0; g->onodes[m].nadj = 0;
        /* a node on an axis-aligned wire joins that conductor: grounded to
         * it like a node on the wall, its charge handed to the grid */
        for (int w = 0; w < g->n_wires; w++)
            if (on_axis_wire(&g->wires[w], g->onodes[m].p)) g->onodes[m].grounded = 1;
    }
    for (int w = 0; w < g->n_owires; w++)
        for (int s = g->owires[w].seg0; s < g->owires[w].seg0 + g->owires[w].nseg; s++) {
            orc_oseg *S = &g->osegs[s];
            /* radius at which the grid sees the segment's current: the
             * bilinear spread of its centre over the line lattice of its
             * dominant axis */
            int u = 0;
            for (int v = 1; v < 3; v++) if (fabs(S->t[v]) > fabs(S->t[u])) u = v;
            int v1 = (u + 1) % 3, v2 = (u + 2) % 3;
            double f1 = S->c[v1] - floor(S->c[v1]), f2 = S->c[v2] - floor(S->c[v2]);
            double w00 = (1 - f1) * (1 - f2), w10 = f1 * (1 - f2), w01 = (1 - f1) * f2, w11 = f1 * f2;
            double S2 = 2.0 * ((w00 * w10 + w01 * w11 + w00 * w01 + w10 * w11) * 0.25 + (w00 * w11 + w10 * w01) / M_PI);
            double R = dx * r0 * exp(2.0 * M_PI * S2);
            double a = g->owires[w].radius;
            S->lam = log(R / a);
            if (!(S->lam > 0.0)) return -1;
            int ci[3];
            for (int q = 0; q < 3; q++) {
                ci[q] = (int)floor(S->c[q]);
                if (ci[q] > nn[q] - 1) ci[q] = nn[q] - 1;
            }
            double Lp = ORC_MU0 * cell_mu(g, ci[0], ci[1], ci[2]) * S->lam / (2.0 * M_PI);
            S->cI = r32(g, dt / Lp);
            S->R = 0.0;
            for (int q = 0; q < g->n_osrcs; q++)
                if (g->osrcs[q].seg == s) S->R += g->osrcs[q].r;
            S->nu = 0.0;
            for (int q = 0; q < 3; q++) S->nu += S->t[q] * S->t[q] * cpml_rate(g, q, S->c[q]);
            double k = 0.5 * dt * (S->R / (Lp * S->dl) + S->nu);
            S->rk = r32(g, (1.0 - k) / (1.0 + k));
            S->rd = r32(g, 1.0 / (1.0 + k));
            /* charge-conserving coupling: the path a -> b split at the cell
             * faces it crosses; each piece inside one cell spreads its
             * displacement over the cell's 12 edges with the weights under
             * which the grid divergence equals the move of a unit charge
             * between the trilinear node weights of its two ends */
            S->ne = 0;
            const double *pa = g->onodes[S->a].p, *pb = g->onodes[S->b].p;
            double cut[8];
            int ncut = 0;
            cut[ncut++] = 0.0;
            for (int q = 0; q < 3; q++) {
                double lo = pa[q] < pb[q] ? pa[q] : pb[q], hi = pa[q] < pb[q] ? pb[q] : pa[q];
                for (double x = floor(lo) + 1.0; x < hi; x += 1.0) {
                    if (ncut >= 7) return -1;
                    cut[ncut++] = (x - pa[q]) / (pb[q] - pa[q]);
                }
            }
            cut[ncut++] = 1.0;
            for (int x = 1; x < ncut; x++)          /* sort the crossing fractions */
                for (int y = x; y > 0 && cut[y] < cut[y - 1]; y--) { double t = cut[y]; cut[y] = cut[y - 1]; cut[y - 1] = t; }
            for (int piece = 0; piece + 1 < ncut; piece++) {
                double u0 = cut[piece], u1 = cut[piece + 1];
                if (!(u1 > u0)) continue;
                double mid[3], dd[3], fr[3];
                int cell[3];
                for (int q = 0; q < 3; q++) {
                    double x0 = pa[q] + u0 * (pb[q] - pa[q]), x1 = pa[q] + u1 * (pb[q] - pa[q]);
                    mid[q] = 0.5 * (x0 + x1);
                    dd[q] = x1 - x0;
                    cell[q] = (int)floor(mid[q]);
                    if (cell[q] > nn[q] - 1) cell[q] = nn[q] - 1;
                    fr[q] = mid[q] - cell[q];
                }
                for (int c = 0; c < 3; c++) {
                    if (dd[c] == 0.0) continue;
                    int v1 = (c + 1) % 3, v2 = (c + 2) % 3;
                    for (int corner = 0; corner < 4; corner++) {
                        int d1 = corner & 1, d2 = corner >> 1;
                        double w1 = d1 ? fr[v1] : 1.0 - fr[v1], w2 = d2 ? fr[v2] : 1.0 - fr[v2];
                        double wt = dd[c] * (w1 * w2 + (d1 == d2 ? 1.0 : -1.0) * dd[v1] * dd[v2] / 12.0);
                        int id[3];
                        id[c] = cell[c];
                        id[v1] = cell[v1] + d1;
                        id[v2] = cell[v2] + d2;
                        if (id[c] < 0 || id[c] > nn[c] - 1 || id[v1] < 1 || id[v1] > nn[v1] - 1 || id[v2] < 1 ||
                            id[v2] > nn[v2] - 1 || wt == 0.0)
                            continue;
                        size_t qi = IDX(g, id[0], id[1], id[2]);
                        int e = 0;
                        while (e < S->ne && !(S->comp[e] == c && S->q[e] == qi)) e++;
                        if (e == S->ne) {
                            if (S->ne >= ORC_OW_EDGES) return -1;
                            S->ne++;
                            S->comp[e] = c;
                            S->q[e] = qi;
                            S->W[e] = 0.0;
                        }
                        S->W[e] += wt;
                    }
                }
            }
            for (int e = 0; e < S->ne; e++) {
                S->wg[e] = r32(g, S->W[e] * dx / S->dl);
                S->ws[e] = r32(g, (double)g->cb[S->comp[e]][S->q[e]] * S->W[e] / dx);
            }
            orc_onode *A = &g->onodes[S->a], *Bn = &g->onodes[S->b];
            A->dlm += 0.5 * S->dl; Bn->dlm += 0.5 * S->dl;
            A->lam_sum += S->lam; Bn->lam_sum += S->lam;
            A->nu_sum += S->nu; Bn->nu_sum += S->nu;
            A->nadj++; Bn->nadj++;
        }
    for (int m = 0; m < g->n_onodes; m++) {
        orc_onode *nd = &g->onodes[m];
        int ci[3];
        for (int q = 0; q < 3; q++) {
            ci[q] = (int)floor(nd->p[q]);
            if (ci[q] > nn[q] - 1) ci[q] = nn[q] - 1;
        }
        int mat = g->mat[CELL(g, ci[0], ci[1], ci[2])];
        double eps = ORC_EPS0 * g->m_eps[mat], sig = g->m_sig[mat];
        double lam = nd->lam_sum / nd->nadj;
        double K = lam / (2.0 * M_PI * nd->dlm);
        /* the CPML's loss acts as an extra conductance eps nu */
        double sig_eff = sig + eps * nd->nu_sum / nd->nadj;
        nd->K = r32(g, K);
        nd->e0 = r32(g, eps);
        nd->cs = r32(g, dt * sig_eff / 2.0);
        for (int p = 0; p < ORC_MAXP; p++) {
            double de = g->m_deps[mat][p], tau = g->m_tau[mat][p];
            nd->pa[p] = de > 0 ? r32(g, (2.0 * tau - dt) / (2.0 * tau + dt)) : 0.0;
            nd->pb[p] = de > 0 ? r32(g, dt * ORC_EPS0 * de / (2.0 * tau + dt)) : 0.0;
        }
        nd->cV = K / eps;
    }
    g->oI = (double *)calloc(g->n_osegs > 0 ? g->n_osegs : 1, sizeof(double));
    g->oQ = (double *)calloc(g->n_onodes > 0 ? g->n_onodes : 1, sizeof(double));
    g->oV = (double *)calloc(g->n_onodes > 0 ? g->n_onodes : 1, sizeof(double));
    g->oP = (double *)calloc((size_t)(g->n_onodes > 0 ? g->n_onodes : 1) * ORC_MAXP, sizeof(double));
    return 0;
}

int orc_finalize(orc_grid *g, int max_steps)
{
    if (g->finalized) return -8;
    if (max_steps < 0) return -1;
    int nx = g->nx, ny = g->ny, nz = g->nz;
    size_t N = g->ntot;
    /* 1. per-edge eps, sigma (mean over the 4 cells around the edge) and
     *    per-face mu (mean over the 2 cells on either side) */
    double *eps[3], *sig[3], *mu[3];
    uint8_t *pec[3];
    double *fac_e[3], *fac_h[3];
    for (int c = 0; c < 3; c++) {
        eps[c] = (double *)calloc(N, sizeof(double));
        sig[c] = (double *)calloc(N, sizeof(double));
        mu[c] = (double *)calloc(N, sizeof(double));
        pec[c] = (uint8_t *)calloc(N, 1);
        fac_e[c] = (double *)malloc(N * sizeof(double));
        fac_h[c] = (double *)malloc(N * sizeof(double));
        for (size_t q = 0; q < N; q++) { fac_e[c][q] = 1.0; fac_h[c][q] = 1.0; }
    }
    for (int k = 0; k <= nz; k++)
        for (int j = 0; j <= ny; j++)
            for (int i = 0; i <= nx; i++) {
                size_t q = IDX(g, i, j, k);
                /* Ex(i+1/2,j,k): cells (i, j-1|j, k-1|k) */
                if (i < nx && j >= 1 && j < ny && k >= 1 && k < nz) {
                    eps[0][q] = 0.25 * (cell_eps(g, i, j - 1, k - 1) + cell_eps(g, i, j, k - 1) +
                                        cell_eps(g, i, j - 1, k) + cell_eps(g, i, j, k));
                    sig[0][q] = 0.25 * (cell_sig(g, i, j - 1, k - 1) + cell_sig(g, i, j, k - 1) +
                                        cell_sig(g, i, j - 1, k) + cell_sig(g, i, j, k));
                }
                /* Ey(i,j+1/2,k): cells (i-1|i, j, k-1|k) */
                if (j < ny && i >= 1 && i < nx && k >= 1 && k < nz) {
                    eps[1][q] = 0.25 * (cell_eps(g, i - 1, j, k - 1) + cell_eps(g, i, j, k - 1) +
                                        cell_eps(g, i - 1, j, k) + cell_eps(g, i, j, k));
                    sig[1][q] = 0.25 * (cell_sig(g, i - 1, j, k - 1) + cell_sig(g, i, j, k - 1) +
                                        cell_sig(g, i - 1, j, k) + cell_sig(g, i, j, k));
                }
                /* Ez(i,j,k+1/2): cells (i-1|i, j-1|j, k) */
                if (k < nz && i >= 1 && i < nx && j >= 1 && j < ny) {
                    eps[2][q] = 0.25 * (cell_eps(g, i - 1, j - 1, k) + cell_eps(g, i, j - 1, k) +
                                        cell_eps(g, i - 1, j, k) + cell_eps(g, i, j, k));
                    sig[2][q] = 0.25 * (cell_sig(g, i - 1, j - 1, k) + cell_sig(g, i, j - 1, k) +
                                        cell_sig(g, i - 1, j, k) + cell_sig(g, i, j, k));
                }
                /* Hx(i,j+1/2,k+1/2): cells i-1 and i */
                if (i >= 1 && i < nx && j < ny && k < nz)
                    mu[0][q] = 0.5 * (cell_mu(g, i - 1, j, k) + cell_mu(g, i, j, k));
                /* Hy(i+1/2,j,k+1/2): cells j-1 and j */
                if (j >= 1 && j < ny && i < nx && k < nz)
                    mu[1][q] = 0.5 * (cell_mu(g, i, j - 1, k) + cell_mu(g, i, j, k));
                /* Hz(i+1/2,j+1/2,k): cells k-1 and k */
                if (k >= 1 && k < nz && i < nx && j < ny)
                    mu[2][q] = 0.5 * (cell_mu(g, i, j, k - 1) + cell_mu(g, i, j, k));
            }
    /* 2. thin wires: on-wire E is PEC; the four radial E at every wire node
     *    (end nodes included) get eps, sigma * m; every H that one of those
     *    radial E reads in its update (the circumferential H of each
     *    segment, the axial H at each node, and the circumferential H just
     *    beyond each end) gets mu / m.  Giving mu/m to every H next to a
     *    modified E keeps each E-H coupling at or below its unmodified
     *    value, which keeps the scheme stable up to S = 1 (radial eps*m next
     *    to an unmodified axial H is not).  Where two wires touch one
     *    component the smaller m (thinner wire) is used once. */
    for (int w = 0; w < g->n_wires; w++) {
        orc_wire *wr = &g->wires[w];
        double m = wire_factor(g, wr->radius);
        int a = wr->axis, b = (a + 1) % 3, c = (a + 2) % 3;
        for (int s = 0; s <= wr->n; s++) {
            int p[3] = {wr->i, wr->j, wr->k};
            p[a] += s;
            /* radial E at node p: E_b at p and p - e_b; E_c at p and p - e_c */
            for (int r = 0; r < 4; r++) {
                int comp = (r < 2) ? b : c;
                int q[3] = {p[0], p[1], p[2]};
                q[comp] -= (r & 1);
                if (!e_interior(g, comp, q)) continue;     /* wall: PEC anyway */
                size_t iq = IDX(g, q[0], q[1], q[2]);
                if (m < fac_e[comp][iq]) fac_e[comp][iq] = m;
                /* the four H this E reads (its curl stencil) */
                int hc[4], hp[4][3];
                e_stencil(comp, q, hc, hp);
                for (int t = 0; t < 4; t++) {
                    size_t ih = IDX(g, hp[t][0], hp[t][1], hp[t][2]);
                    if (m < fac_h[hc[t]][ih]) fac_h[hc[t]][ih] = m;
                }
            }
            /* the on-wire edge E_a(p) of the segment p -> p + e_a is PEC */
            if (s < wr->n) pec[a][IDX(g, p[0], p[1], p[2])] = 1;
        }
    }
    /* 3. coefficients of the semi-implicit update (Eq. fdtdex with the loss
     *    time-averaged) and of Eq. fdtdhx; 1/dx folded in */
    double dt = g->dt, dx = g->dx;
    /* lumped elements and internal resistances: extra eps, sigma per edge */
    double *le[3] = {NULL, NULL, NULL}, *ls[3] = {NULL, NULL, NULL};
    if (g->n_lumps) {
        for (int c = 0; c < 3; c++) { le[c] = (double *)calloc(N, sizeof(double)); ls[c] = (double *)calloc(N, sizeof(double)); }
        for (int l = 0; l < g->n_lumps; l++) {
            const orc_lump *lp = &g->lumps[l];
            size_t q = IDX(g, lp->i, lp->j, lp->k);
            le[lp->axis][q] += lp->e_add;
            ls[lp->axis][q] += lp->s_add;
        }
    }
    if (g->has_debye) {
        for (int c = 0; c < 3; c++) {
            g->eprev[c] = (real *)calloc(N, sizeof(real));
            for (int p = 0; p < ORC_MAXP; p++) {
                g->dcj[c][p] = (real *)calloc(N, sizeof(real));
                g->dk[c][p] = (real *)calloc(N, sizeof(real));
                g->dbe[c][p] = (real *)calloc(N, sizeof(real));
                g->J[c][p] = (real *)calloc(N, sizeof(real));
            }
        }
    }
    for (int c = 0; c < 3; c++) {
        g->ca[c] = (real *)calloc(N, sizeof(real));
        g->cb[c] = (real *)calloc(N, sizeof(real));
        g->db[c] = (real *)calloc(N, sizeof(real));
        for (size_t q = 0; q < N; q++) {
            if (eps[c][q] > 0 && !pec[c][q]) {
                double deps[ORC_MAXP], tau[ORC_MAXP], ca, cb, cj[ORC_MAXP], kk[ORC_MAXP], be[ORC_MAXP];
                if (g->has_debye) {
                    int k = (int)(q / g->sz), j = (int)((q % g->sz) / g->sy), i = (int)(q % g->sy);
                    edge_poles(g, c, i, j, k, deps, tau);
                }
                int disp = e_coefs(g, eps[c][q], sig[c][q], fac_e[c][q], le[c] ? le[c][q] : 0.0,
                                   ls[c] ? ls[c][q] : 0.0, g->has_debye ? deps : NULL, tau, &ca, &cb, cj, kk, be);
                g->ca[c][q] = r32(g, ca);
                g->cb[c][q] = r32(g, cb);
                if (disp)
                    for (int p = 0; p < ORC_MAXP; p++) {
                        g->dcj[c][p][q] = r32(g, cj[p]);
                        g->dk[c][p][q] = r32(g, kk[p]);
                        g->dbe[c][p][q] = r32(g, be[p]);
                    }
            }
            if (mu[c][q] > 0) {
                double mm = ORC_MU0 * mu[c][q] / fac_h[c][q];
                g->db[c][q] = r32(g, dt / (mm * dx));
            }
        }
    }
    /* source factor -cb/dx on each source edge (J = I/dx^2 in Eq. maxwell) */
    g->src_coef = (real *)calloc(g->n_srcs > 0 ? g->n_srcs : 1, sizeof(real));
    for (int s = 0; s < g->n_srcs; s++) {
        orc_src *sr = &g->srcs[s];
        size_t q = IDX(g, sr->i, sr->j, sr->k);
        double cbq;
        if (eps[sr->axis][q] > 0 && !pec[sr->axis][q]) {
            double deps[ORC_MAXP], tau[ORC_MAXP], ca, cj[ORC_MAXP], kk[ORC_MAXP], be[ORC_MAXP];
            if (g->has_debye) edge_poles(g, sr->axis, sr->i, sr->j, sr->k, deps, tau);
            e_coefs(g, eps[sr->axis][q], sig[sr->axis][q], fac_e[sr->axis][q], le[sr->axis] ? le[sr->axis][q] : 0.0,
                    ls[sr->axis] ? ls[sr->axis][q] : 0.0, g->has_debye ? deps : NULL, tau, &ca, &cbq, cj, kk, be);
        } else {
            cbq = 0.0;
        }
        g->src_coef[s] = r32(g, -cbq / dx);
    }
    g->hard_coef = (real *)calloc(g->n_srcs > 0 ? g->n_srcs : 1, sizeof(real));
    for (int s = 0; s < g->n_srcs; s++)
        if (g->srcs[s].hard) g->hard_coef[s] = r32(g, -1.0 / dx);
    for (int c = 0; c < 3; c++) { free(le[c]); free(ls[c]); }
    for (int c = 0; c < 3; c++) { free(eps[c]); free(sig[c]); free(mu[c]); free(pec[c]); free(fac_e[c]); free(fac_h[c]); }
    build_cpml(g);
    if (g->n_owires > 0 && build_owires(g) != 0) return -1;
    g->max_steps = max_steps;
    g->probe_out = (double *)calloc((size_t)(g->n_probes > 0 ? g->n_probes : 1) * (max_steps > 0 ? max_steps : 1), sizeof(double));
    g->finalized = 1;
    return 0;
}

/* ---- field exchange in the cell-owned layout ---- */
int orc_set_field(orc_grid *g, int comp, const double *cells)
{
    if (comp < 0 || comp > 5) return -1;
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++)
                g->f[comp][IDX(g, i, j, k)] = cells[CELL(g, i, j, k)];
    return 0;
}

int orc_get_field(const orc_grid *g, int comp, double *cells)
{
    if (comp < 0 || comp > 5) return -1;
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++)
                cells[CELL(g, i, j, k)] = g->f[comp][IDX(g, i, j, k)];
    return 0;
}

int orc_get_coef(const orc_grid *g, int which, double *cells)
{
    /* which: 0..2 ca_x..z, 3..5 cb_x..z, 6..8 db_x..z */
    if (!g->finalized || which < 0 || which > 8) return -1;
    const real *src = which < 3 ? g->ca[which] : which < 6 ? g->cb[which - 3] : g->db[which - 6];
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++)
                cells[CELL(g, i, j, k)] = src[IDX(g, i, j, k)];
    return 0;
}

/* ---- one time step ---- */

/* one curl term along axis u: plain difference, or in the CPML layer
 * d/kappa + psi with psi <- b psi + c d.  Differences are in field units
 * (1/dx sits in the coefficients), so psi is kept in the same units. */
static inline real term(real dif, real *psi, size_t q, int on, real b, real c, real ki)
{
    if (!on) return dif;
    psi[q] = b * psi[q] + c * dif;
    return dif * ki + psi[q];
}

static void update_h(orc_grid *g)
{
    int nx = g->nx, ny = g->ny, nz = g->nz;
    real *Ex = g->f[EX], *Ey = g->f[EY], *Ez = g->f[EZ];
    real *Hx = g->f[HX], *Hy = g->f[HY], *Hz = g->f[HZ];
    size_t sy = g->sy, sz = g->sz;
    /* Hx(i,j+1/2,k+1/2) += db [dEy/dz - dEz/dy]; i = 0 and nx are normal walls */
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 1; i < nx; i++) {
                size_t q = IDX(g, i, j, k);
                real tz = term(Ey[q + sz] - Ey[q], g->psi[HX][2], q, g->ph_on[2][k], g->ph_b[2][k], g->ph_c[2][k], g->ph_ki[2][k]);
                real ty = term(Ez[q + sy] - Ez[q], g->psi[HX][1], q, g->ph_on[1][j], g->ph_b[1][j], g->ph_c[1][j], g->ph_ki[1][j]);
                Hx[q] += g->db[0][q] * (tz - ty);
            }
    /* Hy(i+1/2,j,k+1/2) += db [dEz/dx - dEx/dz]; j = 0 and ny are walls */
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 1; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t q = IDX(g, i, j, k);
                real tx = term(Ez[q + 1] - Ez[q], g->psi[HY][0], q, g->ph_on[0][i], g->ph_b[0][i], g->ph_c[0][i], g->ph_ki[0][i]);
                real tz = term(Ex[q + sz] - Ex[q], g->psi[HY][2], q, g->ph_on[2][k], g->ph_b[2][k], g->ph_c[2][k], g->ph_ki[2][k]);
                Hy[q] += g->db[1][q] * (tx - tz);
            }
    /* Hz(i+1/2,j+1/2,k) += db [dEx/dy - dEy/dx]; k = 0 and nz are walls */
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 1; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t q = IDX(g, i, j, k);
                real ty = term(Ex[q + sy] - Ex[q], g->psi[HZ][1], q, g->ph_on[1][j], g->ph_b[1][j], g->ph_c[1][j], g->ph_ki[1][j]);
                real tx = term(Ey[q + 1] - Ey[q], g->psi[HZ][0], q, g->ph_on[0][i], g->ph_b[0][i], g->ph_c[0][i], g->ph_ki[0][i]);
                Hz[q] += g->db[2][q] * (ty - tx);
            }
}

/* E^{n+1} += sum_p cj_p J_p^n at node q of component c */
static inline real debye_add(const orc_grid *g, int c, size_t q, real e)
{
    for (int p = 0; p < ORC_MAXP; p++) e += g->dcj[c][p][q] * g->J[c][p][q];
    return e;
}


/* oblique wires, first half: I_s^{n+1/2} from E^n along the segment, the
 * node potentials V_m^n = cV Q_m^n (zero at grounded nodes) and the
 * delta-gap EMFs at t_n */
static void owire_current(orc_grid *g)
{
    double *drive = (double *)calloc(g->n_osegs > 0 ? g->n_osegs : 1, sizeof(double));
    for (int q = 0; q < g->n_osrcs; q++) {
        const orc_osrc *sr = &g->osrcs[q];
        if (g->step < sr->n) drive[sr->seg] += sr->emf[g->step];
    }
    for (int s = 0; s < g->n_osegs; s++) {
        const orc_oseg *S = &g->osegs[s];
        double es = 0.0;
        for (int e = 0; e < S->ne; e++) es += (double)S->wg[e] * g->f[S->comp[e]][S->q[e]];
        const orc_onode *A = &g->onodes[S->a], *B = &g->onodes[S->b];
        double va = A->grounded ? 0.0 : g->oV[S->a];
        double vb = B->grounded ? 0.0 : g->oV[S->b];
        double inc = (double)S->cI * (es - (vb - va) / S->dl + drive[s] / S->dl);
        g->oI[s] = (double)S->rk * g->oI[s] + (double)S->rd * inc;
    }
    free(drive);
}

/* the segment currents in Ampere's law: E^{n+1} -= cb dx J on the coupling
 * edges */
static void owire_inject(orc_grid *g)
{
    for (int s = 0; s < g->n_osegs; s++) {
        const orc_oseg *S = &g->osegs[s];
        for (int e = 0; e < S->ne; e++) g->f[S->comp[e]][S->q[e]] -= (double)S->ws[e] * g->oI[s];
    }
}

/* second half: Q_m^{n+1} from the net segment current into each node at
 * t_{n+1/2}, with the medium's relaxation */
static void owire_charge(orc_grid *g)
{
    if (g->n_onodes == 0) return;
    double *net = (double *)calloc(g->n_onodes, sizeof(double));
    for (int s = 0; s < g->n_osegs; s++) {
        net[g->osegs[s].b] += g->oI[s];
        net[g->osegs[s].a] -= g->oI[s];
    }
    for (int m = 0; m < g->n_onodes; m++) {
        const orc_onode *nd = &g->onodes[m];
        if (nd->grounded) { g->oQ[m] = 0.0; g->oV[m] = 0.0; continue; }
        /* V^{n+1} from K Q^{n+1} = e0 V^{n+1} + sum_p P_p^{n+1} with the
         * charge and polarisation updates substituted */
        double *P = g->oP + (size_t)m * ORC_MAXP;
        double V = g->oV[m], spb = 0.0, spa = 0.0;
        for (int p = 0; p < ORC_MAXP; p++) { spb += nd->pb[p]; spa += (double)nd->pa[p] * P[p]; }
        double Vn = ((double)nd->K * (g->oQ[m] + g->dt * net[m]) - ((double)nd->cs + spb) * V - spa) /
                    ((double)nd->e0 + spb + (double)nd->cs);
        for (int p = 0; p < ORC_MAXP; p++) P[p] = (double)nd->pa[p] * P[p] + (double)nd->pb[p] * (Vn + V);
        g->oQ[m] += g->dt * net[m] - (double)nd->cs / (double)nd->K * (Vn + V);
        g->oV[m] = Vn;
    }
    free(net);
}

static void update_e(orc_grid *g)
{
    int nx = g->nx, ny = g->ny, nz = g->nz;
    real *Ex = g->f[EX], *Ey = g->f[EY], *Ez = g->f[EZ];
    real *Hx = g->f[HX], *Hy = g->f[HY], *Hz = g->f[HZ];
    size_t sy = g->sy, sz = g->sz;
    const int deb = g->has_debye;
    if (deb)
        for (int c = 0; c < 3; c++) memcpy(g->eprev[c], g->f[c], g->ntot * sizeof(real));
    /* Ex(i+1/2,j,k) = ca Ex + cb [dHz/dy - dHy/dz]; j in (0,ny), k in (0,nz) */
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 1; k < nz; k++)
        for (int j = 1; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t q = IDX(g, i, j, k);
                real ty = term(Hz[q] - Hz[q - sy], g->psi[EX][1], q, g->pe_on[1][j], g->pe_b[1][j], g->pe_c[1][j], g->pe_ki[1][j]);
                real tz = term(Hy[q] - Hy[q - sz], g->psi[EX][2], q, g->pe_on[2][k], g->pe_b[2][k], g->pe_c[2][k], g->pe_ki[2][k]);
                Ex[q] = g->ca[0][q] * Ex[q] + g->cb[0][q] * (ty - tz);
                if (deb) Ex[q] = debye_add(g, 0, q, Ex[q]);
            }
    /* Ey(i,j+1/2,k) = ca Ey + cb [dHx/dz - dHz/dx]; i in (0,nx), k in (0,nz) */
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 1; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 1; i < nx; i++) {
                size_t q = IDX(g, i, j, k);
                real tz = term(Hx[q] - Hx[q - sz], g->psi[EY][2], q, g->pe_on[2][k], g->pe_b[2][k], g->pe_c[2][k], g->pe_ki[2][k]);
                real tx = term(Hz[q] - Hz[q - 1], g->psi[EY][0], q, g->pe_on[0][i], g->pe_b[0][i], g->pe_c[0][i], g->pe_ki[0][i]);
                Ey[q] = g->ca[1][q] * Ey[q] + g->cb[1][q] * (tz - tx);
                if (deb) Ey[q] = debye_add(g, 1, q, Ey[q]);
            }
    /* Ez(i,j,k+1/2) = ca Ez + cb [dHy/dx - dHx/dy]; i in (0,nx), j in (0,ny) */
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 1; j < ny; j++)
            for (int i = 1; i < nx; i++) {
                size_t q = IDX(g, i, j, k);
                real tx = term(Hy[q] - Hy[q - 1], g->psi[EZ][0], q, g->pe_on[0][i], g->pe_b[0][i], g->pe_c[0][i], g->pe_ki[0][i]);
                real ty = term(Hx[q] - Hx[q - sy], g->psi[EZ][1], q, g->pe_on[1][j], g->pe_b[1][j], g->pe_c[1][j], g->pe_ki[1][j]);
                Ez[q] = g->ca[2][q] * Ez[q] + g->cb[2][q] * (tx - ty);
                if (deb) Ez[q] = debye_add(g, 2, q, Ez[q]);
            }
    /* oblique-wire currents, then current sources: -cb/dx * I(t_{n+1/2}) on
     * the source edge; then ideal voltage sources force E^{n+1} =
     * -V(t_{n+1}) / dx */
    owire_inject(g);
    for (int s = 0; s < g->n_srcs; s++) {
        orc_src *sr = &g->srcs[s];
        if (sr->hard) continue;
        real I = (g->step < sr->n) ? sr->cur[g->step] : (real)0;
        g->f[sr->axis][IDX(g, sr->i, sr->j, sr->k)] += g->src_coef[s] * I;
    }
    for (int s = 0; s < g->n_srcs; s++) {
        orc_src *sr = &g->srcs[s];
        if (!sr->hard) continue;
        real V = (g->step < sr->n) ? sr->cur[g->step] : (real)0;
        g->f[sr->axis][IDX(g, sr->i, sr->j, sr->k)] = g->hard_coef[s] * V;
    }
    /* PEC walls: tangential E on the six faces is zero (the update loops
     * never touch those entries; they are cleared in case the caller set
     * them) */
#pragma omp parallel for schedule(static)
    for (int k = 0; k <= nz; k++)
        for (int j = 0; j <= ny; j++)
            for (int i = 0; i <= nx; i++) {
                size_t q = IDX(g, i, j, k);
                if (j == 0 || j == ny || k == 0 || k == nz) Ex[q] = 0.0;
                if (i == 0 || i == nx || k == 0 || k == nz) Ey[q] = 0.0;
                if (i == 0 || i == nx || j == 0 || j == ny) Ez[q] = 0.0;
            }
    /* polarisation currents to t_{n+1} from the final E^{n+1} (sources
     * included): J_p^{n+1} = k_p J_p^n + be_p (E^{n+1} - E^n) */
    if (deb)
        for (int c = 0; c < 3; c++)
            for (int p = 0; p < ORC_MAXP; p++) {
                real *Jp = g->J[c][p];
                const real *kk = g->dk[c][p], *be = g->dbe[c][p], *e1 = g->f[c], *e0 = g->eprev[c];
#pragma omp parallel for schedule(static)
                for (size_t q = 0; q < g->ntot; q++) Jp[q] = kk[q] * Jp[q] + be[q] * (e1[q] - e0[q]);
            }
}

/* set the polarisation current J_p^n (E time level) of pole p of E component c
 * (cell-owned layout); only after finalize, on a grid with Debye media */
int orc_set_debye_current(orc_grid *g, int comp, int pole, const double *cells)
{
    if (!g->finalized || !g->has_debye || comp < 0 || comp > 2 || pole < 0 || pole >= ORC_MAXP) return -1;
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++)
                g->J[comp][pole][IDX(g, i, j, k)] = cells[CELL(g, i, j, k)];
    return 0;
}

/* polarisation current of pole p of E component c, cell-owned layout */
int orc_get_debye_current(const orc_grid *g, int comp, int pole, double *cells)
{
    if (comp < 0 || comp > 2 || pole < 0 || pole >= ORC_MAXP) return -1;
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++)
                cells[CELL(g, i, j, k)] = g->has_debye ? g->J[comp][pole][IDX(g, i, j, k)] : 0.0;
    return 0;
}

static double probe_value(const orc_grid *g, const orc_probe *p)
{
    double dx = g->dx;
    if (p->kind == PROBE_W) return g->oI[p->i];
    if (p->kind == PROBE_WV) return g->onodes[p->i].grounded ? 0.0 : g->oV[p->i];
    if (p->kind == PROBE_E) return g->f[p->axis][IDX(g, p->i, p->j, p->k)];
    if (p->kind == PROBE_H) return g->f[3 + p->axis][IDX(g, p->i, p->j, p->k)];
    if (p->kind == PROBE_V) {
        double v = 0.0;
        int q[3] = {p->i, p->j, p->k};
        for (int e = 0; e < p->n_edges; e++) {
            v -= g->f[p->axis][IDX(g, q[0], q[1], q[2])] * dx;
            q[p->axis]++;
        }
        return v;
    }
    /* PROBE_I: circulation of H around the edge, Ampere's law */
    const real *Hx = g->f[HX], *Hy = g->f[HY], *Hz = g->f[HZ];
    int i = p->i, j = p->j, k = p->k;
    if (p->axis == 2)
        return dx * (Hy[IDX(g, i, j, k)] - Hy[IDX(g, i - 1, j, k)] - Hx[IDX(g, i, j, k)] + Hx[IDX(g, i, j - 1, k)]);
    if (p->axis == 0)
        return dx * (Hz[IDX(g, i, j, k)] - Hz[IDX(g, i, j - 1, k)] - Hy[IDX(g, i, j, k)] + Hy[IDX(g, i, j, k - 1)]);
    return dx * (Hx[IDX(g, i, j, k)] - Hx[IDX(g, i, j, k - 1)] - Hz[IDX(g, i, j, k)] + Hz[IDX(g, i - 1, j, k)]);
}

/* advance n full steps: H to n+1/2, oblique-wire currents to n+1/2, record
 * I/H/wire probes, E to n+1 (with the wire and source currents at n+1/2),
 * wire charges to n+1, record V/E probes */
int orc_step(orc_grid *g, int n)
{
    if (!g->finalized) return -8;
    for (int s = 0; s < n; s++) {
        update_h(g);
        owire_current(g);
        for (int p = 0; p < g->n_probes; p++)
            if ((g->probes[p].kind == PROBE_I || g->probes[p].kind == PROBE_H || g->probes[p].kind == PROBE_W) &&
                g->step < g->max_steps)
                g->probe_out[(size_t)p * g->max_steps + g->step] = probe_value(g, &g->probes[p]);
        update_e(g);
        owire_charge(g);
        for (int p = 0; p < g->n_probes; p++)
            if ((g->probes[p].kind == PROBE_V || g->probes[p].kind == PROBE_E || g->probes[p].kind == PROBE_WV) &&
                g->step < g->max_steps)
                g->probe_out[(size_t)p * g->max_steps + g->step] = probe_value(g, &g->probes[p]);
        g->step++;
    }
    return 0;
}

int orc_read_probe(const orc_grid *g, int p, double *out)
{
    if (p < 0 || p >= g->n_probes) return -1;
    memcpy(out, g->probe_out + (size_t)p * g->max_steps, (size_t)g->max_steps * sizeof(double));
    return 0;
}
