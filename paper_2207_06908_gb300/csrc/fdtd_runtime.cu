// fdtd_runtime.cu -- host side of the C ABI declared in include/fdtd.h.
//
// Owns the grid description, turns materials, PEC walls and thin wires into
// per-cell coefficient classes (one byte per cell, <= 256 classes), builds
// the CPML profiles, lays every device buffer out in one arena, and queues
// time steps on the caller's stream, replaying a captured CUDA graph of a
// fixed number of steps where it can.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <array>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include "fdtd.h"
#include "fdtd_internal.h"

namespace {

constexpr double kC0 = 299792458.0;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kMu0 = 1.25663706212e-6;
constexpr double kR0 = 0.23;        // intrinsic radius of a zero-E line, in cells
constexpr int kWatchSteps = 1024;   // default period of the divergence watchdog

struct Wire { int axis, p[3], n; double radius; };
struct Source { int axis, p[3]; std::vector<float> cur; int hard = 0; };   // hard: ideal voltage source
struct Lump { int axis, p[3]; double e_add, s_add; };                      // extra eps (F/m), sigma (S/m) on an edge

// Oblique thin wires: geometry fixed when a wire is added.  Edge shares W
// (cell units, signed) per segment, keyed by E component and edge position.
struct OEdgeH { int comp, q[3]; double W; };
struct OSegH {
    int a, b;                 // end nodes; I flows a -> b
    double dl, lam;           // length (m), ln(R / radius)
    double c[3], t[3];        // centre (node units), direction
    int cell[3];              // cell holding the centre (its mu)
    std::vector<OEdgeH> edges;
};
struct ONodeH { double p[3]; int grounded; };
struct OWireH { int seg0, nseg; };
struct OSrcH { int seg; std::vector<float> emf; double r; };   // r: series resistance (ohm)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

// The z-layer launch and the launch over the planes between the layers
// update disjoint planes from the previous step's buffers only, so one step
// runs them concurrently: the z layers on a side stream forked from the
// step's stream and joined back to it before the source / probe kernel.
struct Fork {
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaError_t init()
    {
        cudaError_t e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
        if (e != cudaSuccess) destroy();
        return e;
    }
    void destroy()
    {
        if (join) cudaEventDestroy(join);
        if (fork) cudaEventDestroy(fork);
        if (side) cudaStreamDestroy(side);
        side = nullptr;
        fork = join = nullptr;
    }
    // launch_a on the side stream and launch_b on s, both after the work
    // already queued on s; s continues after both
    template <class A, class B>
    cudaError_t run(cudaStream_t s, A launch_a, B launch_b) const
    {
        cudaError_t e = cudaEventRecord(fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(side, fork, 0);
        if (e == cudaSuccess) e = launch_a(side);
        if (e == cudaSuccess) e = cudaEventRecord(join, side);
        if (e == cudaSuccess) e = launch_b(s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, join, 0);
        return e;
    }
};

struct fdtd_grid {
    int nx = 0, ny = 0, nz = 0;
    double dx = 0, dt = 0, courant = 0;
    fdtd_cpml cpml{};
    int d = 0;
    cudaStream_t stream = nullptr;
    std::vector<uint8_t> mat;
    std::vector<fdtd_material> table;
    // Debye poles per material index: deps[0..3], tau[4..7] (deps 0 = none)
    std::vector<std::array<double, 2 * fdtd::kMaxPoles>> poles =
        std::vector<std::array<double, 2 * fdtd::kMaxPoles>>(256, {0, 0, 0, 0, 1, 1, 1, 1});
    std::vector<Wire> wires;
    std::vector<Source> srcs;
    std::vector<Lump> lumps;
    std::vector<fdtd::ProbeDesc> probes;
    std::vector<OWireH> owires;
    std::vector<OSegH> osegs;
    std::vector<ONodeH> onodes;
    std::vector<OSrcH> osrcs;
    bool finalized = false;
    int capacity = 0;
    int pitch = 0;
    long long plane = 0;
    // device
    void *arena = nullptr;
    size_t arena_bytes = 0;
    bool own_arena = false;
    float *F[2][6] = {};
    uint8_t *cls = nullptr;
    float *table_d = nullptr;
    int n_classes = 0;
    float *prof[3] = {};
    float *psi[2][fdtd::PSI_COUNT] = {};
    fdtd::SourceDesc *src_d = nullptr;
    float *samples_d = nullptr;
    fdtd::ProbeDesc *probes_d = nullptr;
    float *probe_out = nullptr;
    long long *step_d = nullptr;
    int *work_d = nullptr;          // [2 per launch] step-kernel work counters
    int *err_d = nullptr;           // bounded-wait failure flag
    int *div_d = nullptr;           // watchdog flag: a field held a NaN or an infinity
    int watch = kWatchSteps;        // watchdog period in steps (0 = off)
    int sms = 0;                    // SMs of the grid's device
    fdtd::TmaMaps maps[2];          // TMA descriptors of each input parity
    fdtd::DomainSlot *slot_d = nullptr;   // this grid as a one-domain step launch
    int *item_start_d = nullptr;          // [launch][2]: {0, items}
    int2 *isrc_d = nullptr;               // per current source: {launch, work item} of its edge
    int *order_d = nullptr;               // column tiles in the order a z block hands them out
    std::vector<int> order_pos;           // position of each column tile in that order
    // single-grid steps apply the current sources in the step kernel and read
    // the probes of step n beside step n + 1 (no Debye media, no oblique
    // wires, no ideal voltage sources, at most 32 sources)
    bool fast = false;
    fdtd::DomainSlot slot_h;              // host copy (also read by batches)
    fdtd::EdgeArgs edge_h[2];             // edge-kernel arguments per input parity
    fdtd::PsiGeom pg{};             // staged CPML box geometry
    // The step runs as one launch over the planes between the z layers and,
    // with a CPML, a second launch over the z-layer planes whose shared
    // memory holds the z, x and y auxiliaries at once.  Both read only the
    // input buffers and write disjoint planes.
    struct LaunchCfg {
        int zlo, zhi, zlo2, zhi2, kz, nitems, grid, region, ox, oy, zxy, nh;
        int *work;
    } lc[2] = {};
    int n_launch = 0;
    int ncx = 0, ncy = 0;
    int block = 0;                  // planes per work item (0 = default)
    int *noalloc_err = nullptr;     // error slot of the scratch fdtd_step_noalloc() used
    int parity = 0;
    long step = 0;
    int kz = 0;
    cudaStream_t cap_stream = nullptr;
    Fork fk;                      // concurrent z-layer launch (two-launch grids)
    // Debye media: planes [dz0, dz1) hold every dispersive edge; npoles
    // current arrays per E component over those planes, a record byte per
    // element and the record table
    int npoles = 0, dz0 = 0, dz1 = 0, n_drec = 0;
    float *J = nullptr;
    // oblique wires on the device
    fdtd::OSeg *oseg_d = nullptr;
    int *ochunk_d = nullptr;
    int n_ochunk = 0;
    fdtd::OEdge *oedge_d = nullptr;
    fdtd::OScat *oscat_d = nullptr;
    fdtd::OTerm *oterm_d = nullptr;
    int n_oscat = 0;
    fdtd::ONode *onode_d = nullptr;
    int *oadj_d = nullptr;
    float *oI_d = nullptr, *oQ_d = nullptr, *oV_d = nullptr, *oP_d = nullptr;
    fdtd::OSrc *osrc_d = nullptr;
    float *osamp_d = nullptr;
    uint8_t *dcls_d = nullptr;
    float *dtable_d = nullptr;
    cudaGraphExec_t graph[6] = {};    // captured graphs of 2^k steps (k = 1..5) from parity 0
    std::string err;
};

namespace {

int fail(fdtd_grid *g, int code, const std::string &msg)
{
    if (g) g->err = msg;
    return code;
}

int cuda_fail(fdtd_grid *g, cudaError_t e, const char *what)
{
    return fail(g, FDTD_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// ---- device arena plan -------------------------------------------------
struct Plan {
    size_t field, cls, table, prof[3], psi[fdtd::PSI_COUNT], src, samples, probes, out, step, work, slot, items, isrc,
        order,
        J, dcls, dtable, oseg, ochunk, oedge, oscat, oterm, onode, oadj, oI, oQ, oV, oP, osrc, osamp, total;
};

// poles used by the grid (the largest pole count of a material some cell
// has) and the planes [z0, z1) that hold its dispersive edges: an edge
// averages the cells on its low side, so a cell with poles at plane k makes
// edges of planes k and k + 1 dispersive
int debye_extent(const fdtd_grid *g, int *z0, int *z1)
{
    std::vector<int> np(g->table.size(), 0);
    bool any = false;
    for (size_t m = 0; m < g->table.size(); ++m)
        for (int p = 0; p < fdtd::kMaxPoles; ++p)
            if (g->poles[m][p] > 0) { np[m] = p + 1; any = true; }
    *z0 = *z1 = 0;
    if (!any) return 0;
    int P = 0, kmin = g->nz, kmax = -1;
    const size_t per = (size_t)g->nx * g->ny;
    for (size_t c = 0; c < g->mat.size(); ++c) {
        const int m = g->mat[c];
        if (m < (int)np.size() && np[m] > 0) {
            P = std::max(P, np[m]);
            const int k = (int)(c / per);
            kmin = std::min(kmin, k);
            kmax = std::max(kmax, k);
        }
    }
    *z0 = P ? kmin : 0;
    *z1 = P ? std::min(g->nz, kmax + 2) : 0;
    return P;
}

// a grid whose field arrays hold 2^31 elements or more needs 64-bit indices;
// FDTD_WIDE_INDEX=1 in the environment selects them for any single grid
// (the tests compare both instantiations on small grids)
bool grid_is_wide(const fdtd_grid *g)
{
    static const bool forced = [] {
        const char *v = std::getenv("FDTD_WIDE_INDEX");
        return v && v[0] == '1';
    }();
    return (double)g->plane * g->nz >= 2147483647.0 || forced;
}

// compact auxiliaries: only their axis's two layers (fdtd_internal.h)
int psi_px(const fdtd_grid *g) { return (2 * g->d + 3) / 4 * 4; }
size_t psi_elems(const fdtd_grid *g, int q)
{
    if (g->d == 0) return 0;
    const size_t d2 = 2 * (size_t)g->d;
    switch (q / 4) {
    case 0: return (size_t)g->nz * g->ny * psi_px(g);
    case 1: return (size_t)g->nz * d2 * g->pitch;
    default: return d2 * (size_t)g->plane;
    }
}

Plan make_plan(const fdtd_grid *g, int capacity)
{
    Plan p{};
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t at = off; off = align_up(off + bytes, 256); return at; };
    const size_t cells = (size_t)g->plane * g->nz;
    p.field = take(12 * cells * sizeof(float));
    p.cls = take(cells);
    p.table = take(fdtd::kMaxClasses * fdtd::kNumCoef * sizeof(float));
    const int n[3] = {g->nx, g->ny, g->nz};
    for (int u = 0; u < 3; ++u) p.prof[u] = take(fdtd::PR_COUNT * (size_t)n[u] * sizeof(float));
    for (int q = 0; q < fdtd::PSI_COUNT; ++q) p.psi[q] = take(2 * psi_elems(g, q) * sizeof(float));
    size_t ns = 0;
    for (auto &s : g->srcs) ns += s.cur.size();
    p.src = take(std::max<size_t>(1, g->srcs.size()) * sizeof(fdtd::SourceDesc));
    p.samples = take(std::max<size_t>(1, ns) * sizeof(float));
    p.probes = take(std::max<size_t>(1, g->probes.size()) * sizeof(fdtd::ProbeDesc));
    p.out = take(std::max<size_t>(1, g->probes.size()) * (size_t)std::max(capacity, 1) * sizeof(float));
    p.step = take(sizeof(long long));
    p.work = take(8 * sizeof(int));
    p.slot = take(sizeof(fdtd::DomainSlot));
    p.items = take(4 * sizeof(int));
    p.isrc = take(std::max<size_t>(1, g->srcs.size()) * sizeof(int2));
    const size_t ncols = (size_t)((g->nx + fdtd::geom::TX - 1) / fdtd::geom::TX) *
                         ((g->ny + fdtd::geom::TY - 1) / fdtd::geom::TY);
    p.order = take(ncols * sizeof(int));
    int z0, z1;
    const int P = debye_extent(g, &z0, &z1);
    const size_t box = (size_t)(z1 - z0) * g->plane;
    p.J = take(std::max<size_t>(1, 3 * (size_t)P * box) * sizeof(float));
    p.dcls = take(std::max<size_t>(1, box));
    p.dtable = take(fdtd::kMaxClasses * fdtd::kDebyeRec * sizeof(float));
    size_t n_edge = 0, n_samp = 0;
    for (const OSegH &sg : g->osegs) n_edge += sg.edges.size();
    for (const OSrcH &sr : g->osrcs) n_samp += sr.emf.size();
    const size_t n_os = std::max<size_t>(1, g->osegs.size()), n_on = std::max<size_t>(1, g->onodes.size());
    p.oseg = take(n_os * sizeof(fdtd::OSeg));
    p.ochunk = take((n_os + 1) * sizeof(int));
    p.oedge = take(std::max<size_t>(1, n_edge) * sizeof(fdtd::OEdge));
    p.oscat = take(std::max<size_t>(1, n_edge) * sizeof(fdtd::OScat));
    p.oterm = take(std::max<size_t>(1, n_edge) * sizeof(fdtd::OTerm));
    p.onode = take(n_on * sizeof(fdtd::ONode));
    p.oadj = take(2 * n_os * sizeof(int));
    p.oI = take(n_os * sizeof(float));
    p.oQ = take(n_on * sizeof(float));
    p.oV = take(n_on * sizeof(float));
    p.oP = take(4 * n_on * sizeof(float));
    p.osrc = take(std::max<size_t>(1, g->osrcs.size()) * sizeof(fdtd::OSrc));
    p.osamp = take(std::max<size_t>(1, n_samp) * sizeof(float));
    p.total = off;
    return p;
}

// ---- coefficient classes -----------------------------------------------
// Cell (i,j,k) owns Ex(i+1/2,j,k) Ey(i,j+1/2,k) Ez(i,j,k+1/2) and
// Hx(i,j+1/2,k+1/2) Hy(i+1/2,j,k+1/2) Hz(i+1/2,j+1/2,k).
using Tuple = std::array<uint32_t, fdtd::kNumCoef>;

uint64_t key(int comp, long long cell) { return ((uint64_t)comp << 56) | (uint64_t)cell; }

struct WireMods {
    std::unordered_map<uint64_t, double> fe, fh;   // (component, cell) -> factor
    std::unordered_map<uint64_t, char> pec;         // (E component, cell)
    std::unordered_map<uint64_t, std::pair<double, double>> lump;   // (E component, cell) -> extra eps, sigma
    std::vector<uint8_t> touched;                   // per cell: any entry above
};

bool e_updated(const fdtd_grid *g, int comp, const int q[3])
{
    const int n[3] = {g->nx, g->ny, g->nz};
    for (int u = 0; u < 3; ++u) {
        if (u == comp) { if (q[u] < 0 || q[u] >= n[u]) return false; }
        else if (q[u] < 1 || q[u] > n[u] - 1) return false;
    }
    return true;
}

long long cell_of(const fdtd_grid *g, const int q[3]) { return ((long long)q[2] * g->ny + q[1]) * g->nx + q[0]; }

void set_min(std::unordered_map<uint64_t, double> &m, uint64_t k, double v)
{
    auto it = m.find(k);
    if (it == m.end() || v < it->second) m[k] = v;
}

// Thin wires (Sec. 2.3): the on-wire E edges are PEC; the radial E at each
// wire node take eps, sigma * m; every H such a radial E reads in its update
// takes mu / m (this keeps every E-H coupling at or below its unmodified
// size, so S <= 1 stays stable).  The smaller m wins where wires meet.
WireMods wire_mods(const fdtd_grid *g)
{
    WireMods w;
    w.touched.assign((size_t)g->nx * g->ny * g->nz, 0);
    auto touch = [&](const int q[3]) {
        if (q[0] >= 0 && q[1] >= 0 && q[2] >= 0 && q[0] < g->nx && q[1] < g->ny && q[2] < g->nz)
            w.touched[cell_of(g, q)] = 1;
    };
    for (const Lump &l : g->lumps) {
        auto &v = w.lump[key(l.axis, cell_of(g, l.p))];
        v.first += l.e_add;
        v.second += l.s_add;
        touch(l.p);
    }
    for (const Wire &wr : g->wires) {
        const double m = std::log(1.0 / kR0) / std::log(g->dx / wr.radius);
        const int a = wr.axis;
        for (int s = 0; s <= wr.n; ++s) {
            int p[3] = {wr.p[0], wr.p[1], wr.p[2]};
            p[a] += s;
            for (int t = 1; t <= 2; ++t) {
                const int c = (a + t) % 3;            // radial component
                for (int back = 0; back < 2; ++back) {
                    int q[3] = {p[0], p[1], p[2]};
                    q[c] -= back;
                    if (!e_updated(g, c, q)) continue;
                    set_min(w.fe, key(c, cell_of(g, q)), m);
                    touch(q);
                    // E_c reads H_{c+2} at q and q - e_{c+1}, H_{c+1} at q and q - e_{c+2}
                    const int h1 = (c + 2) % 3, h2 = (c + 1) % 3;
                    int r[3];
                    std::memcpy(r, q, sizeof r); set_min(w.fh, key(h1, cell_of(g, r)), m); touch(r);
                    r[(c + 1) % 3] -= 1; set_min(w.fh, key(h1, cell_of(g, r)), m); touch(r);
                    std::memcpy(r, q, sizeof r); set_min(w.fh, key(h2, cell_of(g, r)), m); touch(r);
                    r[(c + 2) % 3] -= 1; set_min(w.fh, key(h2, cell_of(g, r)), m); touch(r);
                }
            }
            if (s < wr.n) {
                w.pec[key(a, cell_of(g, p))] = 1;
                touch(p);
            }
        }
    }
    return w;
}


// ---- oblique thin wires ---------------------------------------------------
// Radius at which the grid itself sees the current of a segment: the line
// lattice of the segment's dominant axis carries it spread bilinearly over
// the four lines around its centre, and on the square lattice the potential
// of a unit line current falls off as ln(r / r0) / (2 pi) with r0 =
// exp(-gamma) / (2 sqrt 2) cells, while lines one spacing apart interact
// 1/4 less and diagonal ones 1/pi less than a line with itself.
double lattice_radius(double dx, const double c[3], const double t[3])
{
    int u = 0;
    for (int v = 1; v < 3; ++v)
        if (std::fabs(t[v]) > std::fabs(t[u])) u = v;
    const double f1 = c[(u + 1) % 3] - std::floor(c[(u + 1) % 3]);
    const double f2 = c[(u + 2) % 3] - std::floor(c[(u + 2) % 3]);
    const double w[4] = {(1 - f1) * (1 - f2), f1 * (1 - f2), (1 - f1) * f2, f1 * f2};   // (0,0) (1,0) (0,1) (1,1)
    const double side = w[0] * w[1] + w[2] * w[3] + w[0] * w[2] + w[1] * w[3];
    const double diag = w[0] * w[3] + w[1] * w[2];
    const double S = 2.0 * (0.25 * side + diag / M_PI);
    return dx * std::exp(-0.57721566490153286) / (2.0 * std::sqrt(2.0)) * std::exp(2.0 * M_PI * S);
}

// Edge shares of the straight path pa -> pb (node units): cut at every cell
// face it crosses; a piece with displacement dd and midpoint fractions fr in
// its cell gives the edge of component c at the two transverse offsets
// (dv, dw) the share dd_c (w_v w_w +- dd_v dd_w / 12) (+ where dv == dw),
// which makes the grid's discrete divergence of the edge currents equal the
// move of a unit charge between the trilinear node weights of the piece's
// ends (the charge-conserving deposition of particle codes).  Edges the E
// update never touches (the walls) are left out.
std::vector<OEdgeH> path_edges(const fdtd_grid *g, const double pa[3], const double pb[3])
{
    std::vector<double> cut{0.0, 1.0};
    for (int a = 0; a < 3; ++a) {
        const double lo = std::min(pa[a], pb[a]), hi = std::max(pa[a], pb[a]);
        for (double x = std::floor(lo) + 1.0; x < hi; x += 1.0) cut.push_back((x - pa[a]) / (pb[a] - pa[a]));
    }
    std::sort(cut.begin(), cut.end());
    const int n[3] = {g->nx, g->ny, g->nz};
    std::map<std::array<int, 4>, double> share;
    for (size_t q = 0; q + 1 < cut.size(); ++q) {
        if (!(cut[q + 1] > cut[q])) continue;
        double dd[3], fr[3];
        int cell[3];
        for (int a = 0; a < 3; ++a) {
            const double x0 = pa[a] + cut[q] * (pb[a] - pa[a]), x1 = pa[a] + cut[q + 1] * (pb[a] - pa[a]);
            const double mid = 0.5 * (x0 + x1);
            dd[a] = x1 - x0;
            cell[a] = std::min((int)std::floor(mid), n[a] - 1);
            fr[a] = mid - cell[a];
        }
        for (int c = 0; c < 3; ++c) {
            if (dd[c] == 0.0) continue;
            const int v = (c + 1) % 3, w = (c + 2) % 3;
            for (int dv = 0; dv < 2; ++dv)
                for (int dw = 0; dw < 2; ++dw) {
                    const double W = dd[c] * ((dv ? fr[v] : 1.0 - fr[v]) * (dw ? fr[w] : 1.0 - fr[w]) +
                                              (dv == dw ? 1.0 : -1.0) * dd[v] * dd[w] / 12.0);
                    int e[3];
                    e[c] = cell[c];
                    e[v] = cell[v] + dv;
                    e[w] = cell[w] + dw;
                    if (W != 0.0 && e_updated(g, c, e)) share[{c, e[0], e[1], e[2]}] += W;
                }
        }
    }
    std::vector<OEdgeH> out;
    for (const auto &kv : share) out.push_back(OEdgeH{kv.first[0], {kv.first[1], kv.first[2], kv.first[3]}, kv.second});
    return out;
}

// Courant number up to which the leapfrog of grid and oblique wires stays
// stable.  Each segment adds to the grid's stiffness a rank-one term
// c_s w_s w_s^T on the edges it couples to (w_s its edge shares); c_s grows
// as the wire thickens (small Lambda = ln(R/a)).  Measured limits of the
// stiffest single case, a wire along a node line (w = one edge of share 1):
// 1/S^2 - 1 = 0.458, 0.243, 0.138, 0.079, 0.039, 0.013 at Lambda = 0.7, 1.0,
// 1.3, 1.6, 2.0, 2.6, close to 1.71 exp(-1.89 Lambda); the bound takes c_s =
// 2.0 exp(-1.89 Lambda_s) and, since segments that share edges (wires
// converging at a sharp angle) add their terms, the largest row sum over
// the edges of the summed terms: 1/S^2 - 1 = max_e sum_s |w_se| |w_s|_1 c_s
// (equal to c_s for a lone segment on a node line).
double wire_courant_limit(const fdtd_grid *g)
{
    std::map<std::pair<int, long long>, double> row;   // (component, cell) -> row sum
    for (const OSegH &sg : g->osegs) {
        double l1 = 0.0;
        for (const OEdgeH &e : sg.edges) l1 += std::fabs(e.W);
        const double c = 2.0 * std::exp(-1.89 * sg.lam);
        for (const OEdgeH &e : sg.edges) {
            const long long cell = ((long long)e.q[2] * g->ny + e.q[1]) * g->nx + e.q[0];
            row[{e.comp, cell}] += std::fabs(e.W) * l1 * c;
        }
    }
    double worst = 0.0;
    for (const auto &kv : row) worst = std::max(worst, kv.second);
    return 1.0 / std::sqrt(1.0 + worst);
}

// CPML attenuation sigma / (kappa eps0) along axis u at position x (cells)
double cpml_rate(const fdtd_grid *g, int u, double x)
{
    if (g->d == 0) return 0.0;
    const int n = u == 0 ? g->nx : (u == 1 ? g->ny : g->nz), d = g->d;
    const double rho = x < d ? d - x : (x > n - d ? x - (n - d) : 0.0);
    if (rho <= 0.0) return 0.0;
    const double r = rho / d;
    const fdtd_cpml &p = g->cpml;
    return p.sigma_max * std::pow(r, p.order) / ((1.0 + (p.kappa_max - 1.0) * std::pow(r, p.order)) * kEps0);
}

struct WireDev {
    std::vector<int> chunk;          // first segment of each gather chunk, then n_seg
    std::vector<fdtd::OSeg> seg;
    std::vector<fdtd::OEdge> edge;
    std::vector<fdtd::OScat> scat;
    std::vector<fdtd::OTerm> term;
    std::vector<fdtd::ONode> node;
    std::vector<int> adj;
    std::vector<fdtd::OSrc> src;
    std::vector<float> samples;
};

// in-cell parameters (Sec. 2.3 oblique wires, per unit length: L' = mu ln(R/a)
// / (2 pi) on a segment, C' = 2 pi eps / ln(R/a) and G' = 2 pi sigma /
// ln(R/a) at a node, with the node's ln(R/a) the mean of its segments') and
// coupling coefficients; cb of each coupling edge from the class table.
// The scatter is transposed to one entry per coupled edge with its segments
// in order, and each segment lists its sources, so the device sums in a
// fixed order.
WireDev wire_device(const fdtd_grid *g, const std::vector<uint8_t> &cls, const std::vector<float> &table)
{
    WireDev d;
    const double dx = g->dx, dt = g->dt;
    const int n[3] = {g->nx, g->ny, g->nz};
    auto material = [&](const int c[3]) -> const fdtd_material & {
        return g->table[g->mat[((size_t)c[2] * g->ny + c[1]) * g->nx + c[0]]];
    };
    std::vector<double> lam(g->onodes.size(), 0.0), dlm(g->onodes.size(), 0.0), nu(g->onodes.size(), 0.0);
    std::vector<int> deg(g->onodes.size(), 0);
    std::vector<std::vector<int>> adj(g->onodes.size());
    std::vector<std::vector<int>> seg_src(g->osegs.size());
    for (size_t q = 0; q < g->osrcs.size(); ++q) seg_src[g->osrcs[q].seg].push_back((int)q);
    std::map<std::pair<int, long long>, std::vector<fdtd::OTerm>> scat;   // (comp, idx) -> terms
    for (size_t s = 0; s < g->osegs.size(); ++s) {
        const OSegH &sg = g->osegs[s];
        const double Lp = kMu0 * material(sg.cell).mu_r * sg.lam / (2.0 * M_PI);
        fdtd::OSeg o{};
        o.a = sg.a;
        o.b = sg.b;
        o.e0 = (int)d.edge.size();
        o.ne = (int)sg.edges.size();
        o.cI = (float)(dt / Lp);
        o.cIV = (float)(dt / (Lp * sg.dl));
        double R = 0.0;
        for (int q : seg_src[s]) R += g->osrcs[q].r;
        // inside the CPML the wire is a matched lossy line, R'/L' = G'/C' = nu
        double nu_s = 0.0;
        for (int u = 0; u < 3; ++u) nu_s += sg.t[u] * sg.t[u] * cpml_rate(g, u, sg.c[u]);
        const double k = 0.5 * dt * (R / (Lp * sg.dl) + nu_s);
        o.rk = (float)((1.0 - k) / (1.0 + k));
        o.rd = (float)(1.0 / (1.0 + k));
        for (const OEdgeH &e : sg.edges) {
            const long long idx = (long long)e.q[2] * g->plane + (long long)e.q[1] * g->pitch + e.q[0];
            const double cb = table[(size_t)cls[idx] * fdtd::kNumCoef + 3 + e.comp];
            d.edge.push_back(fdtd::OEdge{idx, e.comp, (float)(e.W * dx / sg.dl)});
            scat[{e.comp, idx}].push_back(fdtd::OTerm{(int)s, (float)(cb * e.W / dx)});
        }
        o.s0 = (int)d.src.size();
        o.ns = (int)seg_src[s].size();
        for (int q : seg_src[s]) {
            const OSrcH &sr = g->osrcs[q];
            d.src.push_back(fdtd::OSrc{(int)sr.emf.size(), (long long)d.samples.size(), o.cIV});
            d.samples.insert(d.samples.end(), sr.emf.begin(), sr.emf.end());
        }
        d.seg.push_back(o);
        for (int end = 0; end < 2; ++end) {
            const int m = end ? sg.b : sg.a;
            lam[m] += sg.lam;
            nu[m] += nu_s;
            dlm[m] += 0.5 * sg.dl;
            deg[m] += 1;
            adj[m].push_back((int)(s << 1) | end);
        }
    }
    for (size_t s = 0; s < d.seg.size(); ++s)
        if (d.chunk.empty() || d.seg[s].e0 + d.seg[s].ne - d.seg[d.chunk.back()].e0 > fdtd::kWireChunk)
            d.chunk.push_back((int)s);
    d.chunk.push_back((int)d.seg.size());
    for (auto &kv : scat) {
        d.scat.push_back(fdtd::OScat{kv.first.second, kv.first.first, (int)d.term.size(), (int)kv.second.size()});
        d.term.insert(d.term.end(), kv.second.begin(), kv.second.end());
    }
    for (size_t m = 0; m < g->onodes.size(); ++m) {
        const ONodeH &nd = g->onodes[m];
        int c[3];
        for (int a = 0; a < 3; ++a) c[a] = std::min((int)std::floor(nd.p[a]), n[a] - 1);
        const fdtd_material &mt = material(c);
        const int mat = g->mat[((size_t)c[2] * g->ny + c[1]) * g->nx + c[0]];
        const double eps = kEps0 * mt.eps_r;
        fdtd::ONode o{};
        // K Q = e0 V + sum_p P_p; the CPML's loss acts as an extra conductance eps nu
        o.K = (float)(lam[m] / deg[m] / (2.0 * M_PI * dlm[m]));
        o.e0 = (float)eps;
        o.cs = (float)(dt * (mt.sigma + eps * nu[m] / deg[m]) / 2.0);
        for (int p2 = 0; p2 < fdtd::kMaxPoles; ++p2) {
            const double de = g->poles[mat][p2], tau = g->poles[mat][fdtd::kMaxPoles + p2];
            o.pa[p2] = de > 0 ? (float)((2.0 * tau - dt) / (2.0 * tau + dt)) : 0.f;
            o.pb[p2] = de > 0 ? (float)(dt * kEps0 * de / (2.0 * tau + dt)) : 0.f;
        }
        o.grounded = nd.grounded;
        o.adj0 = (int)d.adj.size();
        o.nadj = (int)adj[m].size();
        d.adj.insert(d.adj.end(), adj[m].begin(), adj[m].end());
        d.node.push_back(o);
    }
    return d;
}

struct Coefs {
    const fdtd_grid *g;
    const WireMods *w;
    // e_add, s_add: lumped capacitance / dx and conductance / dx of the edge,
    // added after the wire factor
    double e_coef(double eps_r, double sigma, double f, double e_add, double s_add, double *cb) const
    {
        const double e = kEps0 * eps_r * f + e_add;
        const double s = sigma * f + s_add;
        const double a = s * g->dt / (2.0 * e);
        *cb = g->dt / (e * g->dx) / (1.0 + a);
        return (1.0 - a) / (1.0 + a);
    }
    // dispersive edge (ADE form): with eps, sigma and every deps scaled by
    // the wire factor f, D = 2 eps + sum beta_p + sigma dt,
    // ca = (2 eps + sum beta_p - sigma dt) / D, cb = 2 dt / (D dx),
    // cj_p = -dt (1 + k_p) / D, k_p = (2 tau_p - dt) / (2 tau_p + dt),
    // be_p = beta_p / dt, beta_p = 2 eps0 deps_p dt / (2 tau_p + dt)
    double e_coef_debye(double eps_r, double sigma, double f, double e_add, double s_add, const double *deps,
                        const double *tau, double *cb, double *cj, double *kk, double *be) const
    {
        const double dt = g->dt;
        const double e = kEps0 * eps_r * f + e_add, s = sigma * f + s_add;
        double beta[fdtd::kMaxPoles], sb = 0.0;
        for (int p = 0; p < fdtd::kMaxPoles; ++p) {
            beta[p] = 2.0 * kEps0 * deps[p] * f * dt / (2.0 * tau[p] + dt);
            kk[p] = deps[p] > 0 ? (2.0 * tau[p] - dt) / (2.0 * tau[p] + dt) : 0.0;
            sb += beta[p];
        }
        const double D = 2.0 * e + sb + s * dt;
        *cb = 2.0 * dt / (D * g->dx);
        for (int p = 0; p < fdtd::kMaxPoles; ++p) {
            cj[p] = deps[p] > 0 ? -dt * (1.0 + kk[p]) / D : 0.0;
            be[p] = deps[p] > 0 ? beta[p] / dt : 0.0;
        }
        return (2.0 * e + sb - s * dt) / D;
    }
    // Debye poles of E component c of cell (i,j,k): each pole's deps is the
    // mean over the four cells the edge averages (zero where a cell lacks
    // the pole), its tau the deps-weighted mean over those that have it
    bool e_poles(int c, int i, int j, int k, double *deps, double *tau) const
    {
        int cell[4][3];
        for (int t = 0; t < 4; ++t) {
            const int a = t & 1, b = t >> 1;
            if (c == 0) { cell[t][0] = i; cell[t][1] = j - 1 + a; cell[t][2] = k - 1 + b; }
            else if (c == 1) { cell[t][0] = i - 1 + a; cell[t][1] = j; cell[t][2] = k - 1 + b; }
            else { cell[t][0] = i - 1 + a; cell[t][1] = j - 1 + b; cell[t][2] = k; }
        }
        bool any = false;
        for (int p = 0; p < fdtd::kMaxPoles; ++p) {
            double sd = 0.0, st = 0.0;
            for (int t = 0; t < 4; ++t) {
                const int m = g->mat[((size_t)cell[t][2] * g->ny + cell[t][1]) * g->nx + cell[t][0]];
                sd += g->poles[m][p];
                st += g->poles[m][p] * g->poles[m][fdtd::kMaxPoles + p];
            }
            deps[p] = 0.25 * sd;
            tau[p] = sd > 0 ? st / sd : 1.0;
            any |= deps[p] > 0;
        }
        return any;
    }
    double h_coef(double mu_r, double f) const { return g->dt / (kMu0 * mu_r / f * g->dx); }
    const fdtd_material &M(int i, int j, int k) const
    {
        return g->table[g->mat[((size_t)k * g->ny + j) * g->nx + i]];
    }
    // E component c of cell (i,j,k): mean eps, sigma of its four cells
    void e_mat(int c, int i, int j, int k, double *eps, double *sig) const
    {
        int di[4], dj[4], dk[4];
        for (int t = 0; t < 4; ++t) { di[t] = i; dj[t] = j; dk[t] = k; }
        const int b = (c + 1) % 3, cc = (c + 2) % 3;
        int *D[3] = {di, dj, dk};
        // cells offset by 0/-1 along the two transverse axes
        D[b][1] -= 1; D[b][3] -= 1;
        D[cc][2] -= 1; D[cc][3] -= 1;
        double e = 0, s = 0;
        for (int t = 0; t < 4; ++t) {
            const fdtd_material &m = M(di[t], dj[t], dk[t]);
            e += m.eps_r;
            s += m.sigma;
        }
        *eps = e / 4.0;
        *sig = s / 4.0;
    }
    // H component c of cell (i,j,k): mean mu of the cells on either side
    double h_mat(int c, int i, int j, int k) const
    {
        int q[3] = {i, j, k};
        const double m1 = M(q[0], q[1], q[2]).mu_r;
        q[c] -= 1;
        return 0.5 * (m1 + M(q[0], q[1], q[2]).mu_r);
    }
    // coefficient of E component c at cell q: returns false for PEC.
    // debye (optional, 3 * kMaxPoles doubles {cj, k, be} per pole) is filled
    // for a dispersive edge and zeroed otherwise; *disp tells which
    bool e_of(int c, const int q[3], long long cell, double *ca, double *cb, double *debye = nullptr,
              bool *disp = nullptr) const
    {
        if (debye) for (int t = 0; t < 3 * fdtd::kMaxPoles; ++t) debye[t] = 0.0;
        if (disp) *disp = false;
        if (!e_updated(g, c, q)) { *ca = 0; *cb = 0; return false; }
        double f = 1.0, e_add = 0.0, s_add = 0.0;
        if (w && w->touched[cell]) {
            if (w->pec.count(key(c, cell))) { *ca = 0; *cb = 0; return false; }
            auto it = w->fe.find(key(c, cell));
            if (it != w->fe.end()) f = it->second;
            auto il = w->lump.find(key(c, cell));
            if (il != w->lump.end()) { e_add = il->second.first; s_add = il->second.second; }
        }
        double eps, sig;
        e_mat(c, q[0], q[1], q[2], &eps, &sig);
        double deps[fdtd::kMaxPoles], tau[fdtd::kMaxPoles];
        if (g->npoles && e_poles(c, q[0], q[1], q[2], deps, tau)) {
            double cj[fdtd::kMaxPoles], kk[fdtd::kMaxPoles], be[fdtd::kMaxPoles];
            *ca = e_coef_debye(eps, sig, f, e_add, s_add, deps, tau, cb, cj, kk, be);
            if (debye)
                for (int p = 0; p < fdtd::kMaxPoles; ++p) {
                    debye[3 * p] = cj[p];
                    debye[3 * p + 1] = kk[p];
                    debye[3 * p + 2] = be[p];
                }
            if (disp) *disp = true;
            return true;
        }
        *ca = e_coef(eps, sig, f, e_add, s_add, cb);
        return true;
    }
    double h_of(int c, const int q[3], long long cell) const
    {
        if (q[c] < 1) return 0.0;           // normal H on a wall never changes
        double f = 1.0;
        if (w && w->touched[cell]) {
            auto it = w->fh.find(key(c, cell));
            if (it != w->fh.end()) f = it->second;
        }
        return h_coef(h_mat(c, q[0], q[1], q[2]), f);
    }
    // the cell's coefficient tuple and its Debye record (all zero when no
    // owned E component is dispersive); returns whether the record is used
    bool cell(int i, int j, int k, float out[fdtd::kNumCoef], float rec[fdtd::kDebyeRec]) const
    {
        const int q[3] = {i, j, k};
        const long long c = cell_of(g, q);
        bool any = false;
        for (int comp = 0; comp < 3; ++comp) {
            double ca, cb, d[3 * fdtd::kMaxPoles];
            bool disp = false;
            e_of(comp, q, c, &ca, &cb, d, &disp);
            out[comp] = (float)ca;
            out[3 + comp] = (float)cb;
            out[6 + comp] = (float)h_of(comp, q, c);
            for (int t = 0; t < 3 * fdtd::kMaxPoles; ++t) rec[comp * 3 * fdtd::kMaxPoles + t] = (float)d[t];
            any |= disp;
        }
        return any;
    }
};

int build_classes(fdtd_grid *g, std::vector<uint8_t> &cls, std::vector<float> &table,
                  std::vector<double> &src_cb, std::vector<uint8_t> &dcls, std::vector<float> &dtable,
                  std::vector<std::array<double, 3 * fdtd::kMaxPoles>> &src_debye)
{
    g->npoles = debye_extent(g, &g->dz0, &g->dz1);
    using Rec = std::array<uint32_t, fdtd::kDebyeRec>;
    WireMods w = wire_mods(g);
    Coefs C{g, &w};
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    cls.assign((size_t)g->plane * nz, 0);
    dcls.assign((size_t)g->plane * nz, 0);
    // Slabs of planes in parallel: each numbers its distinct coefficient sets
    // (and Debye records) in first-encounter order and writes those local
    // ids; merging the slabs in order then gives every set the id a single
    // scan in k, j, i order would, whatever the thread count.
    struct Slab {
        std::vector<Tuple> tup;
        std::vector<Rec> rec{Rec{}};        // local record 0: no dispersive component
        bool over_cls = false, over_rec = false;
    };
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int nth = std::max(1, std::min({(int)hw, 32, nz}));
    std::vector<Slab> slabs(nth);
    auto work = [&](int t) {
        Slab &S = slabs[t];
        std::map<Tuple, int> ids;
        std::map<Rec, int> dids{{Rec{}, 0}};
        std::vector<int> uniform_id(g->table.size(), -1), uniform_did(g->table.size(), 0);
        const size_t sx = 1, sy = nx, sz = (size_t)nx * ny;
        for (int k = nz * t / nth; k < nz * (t + 1) / nth; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    const size_t c = ((size_t)k * ny + j) * nx + i;
                    const uint8_t m0 = g->mat[c];
                    // every cell that any owned component averages over
                    const bool uni = i > 0 && j > 0 && k > 0 && !w.touched[c] && g->mat[c - sx] == m0 &&
                                     g->mat[c - sy] == m0 && g->mat[c - sz] == m0 && g->mat[c - sx - sy] == m0 &&
                                     g->mat[c - sx - sz] == m0 && g->mat[c - sy - sz] == m0;
                    int id, did = 0;
                    if (uni && uniform_id[m0] >= 0) {
                        id = uniform_id[m0];
                        did = uniform_did[m0];
                    } else {
                        float v[fdtd::kNumCoef], r[fdtd::kDebyeRec];
                        if (C.cell(i, j, k, v, r)) {
                            Rec key;
                            std::memcpy(key.data(), r, sizeof key);
                            auto it = dids.find(key);
                            if (it == dids.end()) {
                                it = dids.emplace(key, (int)S.rec.size()).first;
                                S.rec.push_back(key);
                            }
                            did = it->second;
                        }
                        Tuple key;
                        std::memcpy(key.data(), v, sizeof key);
                        auto it = ids.find(key);
                        if (it == ids.end()) {
                            it = ids.emplace(key, (int)S.tup.size()).first;
                            S.tup.push_back(key);
                        }
                        id = it->second;
                        if (uni) { uniform_id[m0] = id; uniform_did[m0] = did; }
                    }
                    if (id >= fdtd::kMaxClasses) { S.over_cls = true; return; }
                    if (did >= fdtd::kMaxClasses) { S.over_rec = true; return; }
                    cls[(size_t)k * g->plane + (size_t)j * g->pitch + i] = (uint8_t)id;
                    dcls[(size_t)k * g->plane + (size_t)j * g->pitch + i] = (uint8_t)did;
                }
    };
    {
        std::vector<std::thread> pool;
        for (int t = 1; t < nth; ++t) pool.emplace_back(work, t);
        work(0);
        for (auto &th : pool) th.join();
    }
    std::map<Tuple, int> ids;
    std::map<Rec, int> dids{{Rec{}, 0}};
    table.clear();
    dtable.assign(fdtd::kDebyeRec, 0.f);
    std::vector<std::array<uint8_t, fdtd::kMaxClasses>> remap(nth), dremap(nth);
    for (int t = 0; t < nth; ++t) {
        const Slab &S = slabs[t];
        if (S.over_cls) return fail(g, FDTD_ECLASSES, "more than 256 distinct coefficient classes");
        if (S.over_rec) return fail(g, FDTD_ECLASSES, "more than 255 distinct dispersive-media records");
        for (size_t q = 0; q < S.tup.size(); ++q) {
            auto it = ids.find(S.tup[q]);
            if (it == ids.end()) {
                it = ids.emplace(S.tup[q], (int)ids.size()).first;
                const float *v = reinterpret_cast<const float *>(S.tup[q].data());
                table.insert(table.end(), v, v + fdtd::kNumCoef);
            }
            if (it->second >= fdtd::kMaxClasses)
                return fail(g, FDTD_ECLASSES, "more than 256 distinct coefficient classes");
            remap[t][q] = (uint8_t)it->second;
        }
        for (size_t q = 0; q < S.rec.size(); ++q) {
            auto it = dids.find(S.rec[q]);
            if (it == dids.end()) {
                it = dids.emplace(S.rec[q], (int)dids.size()).first;
                const float *r = reinterpret_cast<const float *>(S.rec[q].data());
                dtable.insert(dtable.end(), r, r + fdtd::kDebyeRec);
            }
            if (it->second >= fdtd::kMaxClasses)
                return fail(g, FDTD_ECLASSES, "more than 255 distinct dispersive-media records");
            dremap[t][q] = (uint8_t)it->second;
        }
    }
    {
        auto relabel = [&](int t) {
            for (int k = nz * t / nth; k < nz * (t + 1) / nth; ++k)
                for (int j = 0; j < ny; ++j) {
                    uint8_t *cr = cls.data() + (size_t)k * g->plane + (size_t)j * g->pitch;
                    uint8_t *dr = dcls.data() + (size_t)k * g->plane + (size_t)j * g->pitch;
                    for (int i = 0; i < nx; ++i) {
                        cr[i] = remap[t][cr[i]];
                        dr[i] = dremap[t][dr[i]];
                    }
                }
        };
        std::vector<std::thread> pool;
        for (int t = 1; t < nth; ++t) pool.emplace_back(relabel, t);
        relabel(0);
        for (auto &th : pool) th.join();
    }
    g->n_classes = (int)ids.size();
    g->n_drec = (int)dids.size();
    src_cb.clear();
    src_debye.clear();
    for (const Source &s : g->srcs) {
        double ca, cb;
        std::array<double, 3 * fdtd::kMaxPoles> d{};
        bool disp = false;
        C.e_of(s.axis, s.p, cell_of(g, s.p), &ca, &cb, d.data(), &disp);
        src_cb.push_back(cb);
        src_debye.push_back(d);
    }
    return FDTD_OK;
}

// ---- CPML profiles (Sec. 2.2, CFS recursive convolution) ----------------
void cpml_point(const fdtd_grid *g, double rho, float *b, float *c, float *ki)
{
    const fdtd_cpml &p = g->cpml;
    const double x = rho / g->d;
    const double sig = p.sigma_max * std::pow(x, p.order);
    const double kap = 1.0 + (p.kappa_max - 1.0) * std::pow(x, p.order);
    const double alp = p.alpha_max * std::pow(1.0 - x, p.alpha_order);
    const double bb = std::exp(-(sig / kap + alp) * g->dt / kEps0);
    const double cc = sig > 0 ? sig * (bb - 1.0) / (sig * kap + kap * kap * alp) : 0.0;
    *b = (float)bb;
    *c = (float)cc;
    *ki = (float)(1.0 / kap);
}

std::vector<float> cpml_profile(const fdtd_grid *g, int n)
{
    using namespace fdtd;
    std::vector<float> pr(PR_COUNT * (size_t)n, 0.f);
    for (int i = 0; i < n; ++i) {
        pr[PR_BE * n + i] = 1.f; pr[PR_KIE * n + i] = 1.f;
        pr[PR_BH * n + i] = 1.f; pr[PR_KIH * n + i] = 1.f;
    }
    if (g->d == 0) return pr;
    const int d = g->d;
    for (int i = 0; i < n; ++i) {
        // E at node i: depth d - i (low side) or i - (n - d) (high side)
        double re = i < d ? d - i : (i > n - d ? i - (n - d) : 0.0);
        if (re > 0) cpml_point(g, re, &pr[PR_BE * n + i], &pr[PR_CE * n + i], &pr[PR_KIE * n + i]);
        // H at node i + 1/2
        double rh = i < d ? d - (i + 0.5) : (i >= n - d ? (i + 0.5) - (n - d) : 0.0);
        if (rh > 0) cpml_point(g, rh, &pr[PR_BH * n + i], &pr[PR_CH * n + i], &pr[PR_KIH * n + i]);
    }
    return pr;
}

fdtd::StepArgs step_args(const fdtd_grid *g, int parity, int launch)
{
    fdtd::StepArgs a{};
    a.nx = g->nx; a.ny = g->ny; a.nz = g->nz;
    a.pitch = g->pitch; a.plane = g->plane;
    for (int c = 0; c < 3; ++c) {
        a.Ein[c] = g->F[parity][c];
        a.Hin[c] = g->F[parity][3 + c];
        a.Eout[c] = g->F[1 - parity][c];
        a.Hout[c] = g->F[1 - parity][3 + c];
    }
    a.cls = g->cls;
    a.table = g->table_d;
    a.n_classes = g->n_classes;
    a.d = g->d;
    for (int u = 0; u < 3; ++u) a.prof[u] = g->prof[u];
    for (int q = 0; q < fdtd::PSI_COUNT; ++q) {
        a.psi_in[q] = g->psi[parity][q];
        a.psi_out[q] = g->psi[1 - parity][q];
    }
    a.px = psi_px(g);
    const auto &L = g->lc[launch];
    a.kz = L.kz;
    a.zlo = L.zlo;
    a.zhi = L.zhi;
    a.zlo2 = L.zlo2;
    a.zhi2 = L.zhi2;
    a.ncx = g->ncx;
    a.ncy = g->ncy;
    a.nitems = L.nitems;
    a.pg = g->pg;
    a.region = L.region;
    a.ox = L.ox;
    a.oy = L.oy;
    a.zxy = L.zxy;
    a.col_order = g->order_d;
    a.bounds = g->work_d + 6;
    return a;
}

fdtd::EdgeArgs edge_args(const fdtd_grid *g, int parity)
{
    fdtd::EdgeArgs e{};
    e.nx = g->nx; e.ny = g->ny; e.nz = g->nz;
    e.pitch = g->pitch; e.plane = g->plane;
    e.dx = (float)g->dx;
    e.dt = (float)g->dt;
    for (int c = 0; c < 3; ++c) {
        e.E[c] = g->F[1 - parity][c];
        e.H[c] = g->F[1 - parity][3 + c];
    }
    e.src = g->src_d;
    e.n_src = (int)g->srcs.size();
    e.samples = g->samples_d;
    e.probes = g->probes_d;
    e.n_probes = (int)g->probes.size();
    e.probe_out = g->probe_out;
    e.capacity = g->capacity;
    e.step = g->step_d;
    e.J = g->npoles ? g->J : nullptr;
    e.jstride = (long long)(g->dz1 - g->dz0) * g->plane;
    e.npoles = g->npoles;
    for (int c = 0; c < 3; ++c) e.Ein[c] = g->F[parity][c];
    e.w.seg = g->oseg_d;
    e.w.n_seg = (int)g->osegs.size();
    e.w.chunk = g->ochunk_d;
    e.w.n_chunk = g->n_ochunk;
    e.w.edge = g->oedge_d;
    e.w.scat = g->oscat_d;
    e.w.n_scat = g->n_oscat;
    e.w.term = g->oterm_d;
    e.w.node = g->onode_d;
    e.w.n_node = (int)g->onodes.size();
    e.w.adj = g->oadj_d;
    e.w.I = g->oI_d;
    e.w.Q = g->oQ_d;
    e.w.V = g->oV_d;
    e.w.P = g->oP_d;
    e.wire_done = g->npoles > 0 && !g->osegs.empty();
    e.w.src = g->osrc_d;
    e.w.samples = g->osamp_d;
    e.step_t = 0;
    e.advance = 1;
    e.skip_src = 0;
    e.bounds = g->work_d + 6;
    return e;
}

bool has_edge_work(const fdtd_grid *g) { return !g->srcs.empty() || !g->probes.empty() || !g->osegs.empty(); }

fdtd::DebyeArgs debye_args(const fdtd_grid *g, int parity)
{
    fdtd::DebyeArgs a{};
    for (int c = 0; c < 3; ++c) {
        a.Ein[c] = g->F[parity][c];
        a.Eout[c] = g->F[1 - parity][c];
    }
    a.J = g->J;
    a.jstride = (long long)(g->dz1 - g->dz0) * g->plane;
    a.npoles = g->npoles;
    a.dcls = g->dcls_d;
    a.table = g->dtable_d;
    a.n_rec = g->n_drec;
    a.off = (long long)g->dz0 * g->plane;
    return a;
}

fdtd::SingleArgs single_args(const fdtd_grid *g, int parity, int l)
{
    fdtd::SingleArgs one;
    one.m = g->slot_h.m[parity];
    one.a = g->slot_h.a[l][parity];
    return one;
}

// the same, for a single-grid step that applies the current sources in the
// step kernel: step t of a sequence that began at the device counter
fdtd::SingleArgs single_args_fast(const fdtd_grid *g, int parity, int l, int t)
{
    fdtd::SingleArgs one = single_args(g, parity, l);
    one.a.n_isrc = (int)g->srcs.size();
    one.a.isrc_loc = g->isrc_d;
    one.a.src = g->src_d;
    one.a.samples = g->samples_d;
    one.a.step = g->step_d;
    one.a.step_t = t;
    return one;
}

// launch l of one step of this grid alone
fdtd::BatchArgs grid_launch(const fdtd_grid *g, int parity, int l, int *work, int *err)
{
    fdtd::BatchArgs b{};
    b.doms = nullptr;               // single domain: arguments travel in the kernel parameters
    b.item_start = nullptr;
    b.n_domains = 1;
    b.nitems = g->lc[l].nitems;
    b.launch = l;
    b.parity = parity;
    b.work = work;
    b.err = err;
    b.max_classes = g->n_classes;
    b.max_d = g->d;
    b.region = g->lc[l].region;
    b.nh = g->lc[l].nh;
    b.wide = grid_is_wide(g);
    return b;
}

// One step with the current sources in the step kernel (g->fast): step t of
// a sequence whose first step is the device counter's value.  The probes of
// the previous step (t > 0) read that step's output -- this step's input,
// which nothing writes now -- on the side stream beside the step kernels;
// the last step of the sequence (last) reads its own probes after its step
// kernels and advances the counter by t + 1.
cudaError_t enqueue_step_fast(fdtd_grid *g, int parity, cudaStream_t s, int t, bool last)
{
    auto launch = [g, parity, t](int l) {
        return [g, parity, t, l](cudaStream_t st) {
            return fdtd::launch_step(single_args_fast(g, parity, l, t),
                                     grid_launch(g, parity, l, g->lc[l].work, g->err_d), g->lc[l].grid, st);
        };
    };
    const bool prev = t > 0 && !g->probes.empty();
    cudaError_t e = cudaSuccess;
    if (g->fk.side && (g->n_launch == 2 || prev)) {
        auto side = [g, parity, t, prev, &launch](cudaStream_t st) {
            cudaError_t r = g->n_launch == 2 ? launch(1)(st) : cudaSuccess;
            if (r == cudaSuccess && prev) {
                fdtd::EdgeArgs pa = edge_args(g, parity ^ 1);     // step t - 1's output
                pa.n_src = 0;
                pa.skip_src = 1;
                pa.step_t = t - 1;
                pa.advance = 0;
                r = fdtd::launch_edges(pa, st);
            }
            return r;
        };
        e = g->fk.run(s, side, launch(0));
    } else {
        for (int l = 0; l < g->n_launch && e == cudaSuccess; ++l) e = launch(l)(s);
    }
    if (e == cudaSuccess && last) {
        fdtd::EdgeArgs pa = edge_args(g, parity);
        pa.n_src = 0;
        pa.skip_src = 1;
        pa.step_t = t;
        pa.advance = 1;
        e = fdtd::launch_edges(pa, s);
    }
    return e;
}

cudaError_t enqueue_step(fdtd_grid *g, int parity, cudaStream_t s, int t = 0, bool last = true)
{
    if (g->fast) return enqueue_step_fast(g, parity, s, t, last);
    cudaError_t e = cudaSuccess;
    auto launch = [g, parity](int l) {
        return [g, parity, l](cudaStream_t st) {
            return fdtd::launch_step(single_args(g, parity, l), grid_launch(g, parity, l, g->lc[l].work, g->err_d),
                                     g->lc[l].grid, st);
        };
    };
    const bool wires = !g->osegs.empty();
    if (g->fk.side && (g->n_launch == 2 || wires)) {
        // side stream: the oblique wires' gather, then the z-layer launch
        auto side = [g, parity, wires, &launch](cudaStream_t st) {
            cudaError_t r = wires ? fdtd::launch_wire_gather(edge_args(g, parity), st) : cudaSuccess;
            if (r == cudaSuccess && g->n_launch == 2) r = launch(1)(st);
            return r;
        };
        e = g->fk.run(s, side, launch(0));
    } else {
        if (wires) e = fdtd::launch_wire_gather(edge_args(g, parity), s);
        for (int l = 0; l < g->n_launch && e == cudaSuccess; ++l) e = launch(l)(s);
    }
    // in Debye media the wires' currents reach E^{n+1} before the polarisation
    // currents advance from it
    if (e == cudaSuccess && g->npoles && wires) e = fdtd::launch_wire_finish(edge_args(g, parity), s);
    if (e == cudaSuccess && g->npoles) e = fdtd::launch_debye(debye_args(g, parity), s);
    if (e != cudaSuccess) return e;
    if (has_edge_work(g)) e = fdtd::launch_edges(edge_args(g, parity), s);
    return e;
}

// ---- TMA descriptors ----------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 3D tiled map over one array of extent x0 x y0 x z0 with row pitch
// `pitch` elements and y0 rows per plane (x fastest); out-of-range box
// elements read as zero
bool encode_map3(CUtensorMap *m, void *base, CUtensorMapDataType dt, int esize, int x0, int y0, int z0, int pitch,
                 int bx, int by)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)x0, (cuuint64_t)y0, (cuuint64_t)z0};
    cuuint64_t strides[2] = {(cuuint64_t)pitch * esize, (cuuint64_t)pitch * y0 * esize};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    cuuint32_t es[3] = {1, 1, 1};
    return fn(m, dt, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 3D tiled map over one field-shaped array (the fields, the class bytes)
bool encode_map(CUtensorMap *m, void *base, CUtensorMapDataType dt, int esize, const fdtd_grid *g, int bx, int by)
{
    return encode_map3(m, base, dt, esize, g->nx, g->ny, g->nz, g->pitch, bx, by);
}

// Raise (never lower) a step kernel's dynamic shared-memory limit: grids and
// batches created earlier keep launching with their own sizes.
cudaError_t ensure_smem(const void *kernel, int bytes)
{
    static std::mutex lock;
    static std::map<std::pair<int, const void *>, int> set;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> guard(lock);
    int &cur = set[{dev, kernel}];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

int setup_step_kernel(fdtd_grid *g)
{
    using namespace fdtd::geom;
    g->pg = fdtd::step_psi_geom(g->d, g->nx, g->ny);
    for (int p = 0; p < 2; ++p) {
        for (int c = 0; c < 3; ++c) {
            if (!encode_map(&g->maps[p].e[c], g->F[p][c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, g, EBX, EBY) ||
                !encode_map(&g->maps[p].h[c], g->F[p][3 + c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, g, HBX, HBY))
                return fail(g, FDTD_ECUDA, "cuTensorMapEncodeTiled failed for a field");
        }
        if (!encode_map(&g->maps[p].c, g->cls, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, g, CBX, CBY))
            return fail(g, FDTD_ECUDA, "cuTensorMapEncodeTiled failed for the class map");
        if (g->d > 0) {
            using namespace fdtd;
            const auto F32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
            const int w = g->pg.w, hy = g->pg.hy;
            // compact layouts: x [nz][ny][px], y [nz][2d][pitch], z [2d][ny][pitch]
            const int px = psi_px(g), d2 = 2 * g->d;
            struct { CUtensorMap *m; int psi, bx, by; } maps[12] = {
                {&g->maps[p].zh[0], PSI_HX_Z, HBX, HBY}, {&g->maps[p].zh[1], PSI_HY_Z, HBX, HBY},
                {&g->maps[p].ze[0], PSI_EX_Z, TX, TY},   {&g->maps[p].ze[1], PSI_EY_Z, TX, TY},
                {&g->maps[p].xh[0], PSI_HY_X, w, HBY},   {&g->maps[p].xh[1], PSI_HZ_X, w, HBY},
                {&g->maps[p].xe[0], PSI_EY_X, w, HBY},   {&g->maps[p].xe[1], PSI_EZ_X, w, HBY},
                {&g->maps[p].yh[0], PSI_HX_Y, HBX, hy},  {&g->maps[p].yh[1], PSI_HZ_Y, HBX, hy},
                {&g->maps[p].ye[0], PSI_EX_Y, HBX, hy},  {&g->maps[p].ye[1], PSI_EZ_Y, HBX, hy}};
            for (auto &mm : maps) {
                const int axis = mm.psi / 4;
                const bool ok = axis == 0   ? encode_map3(mm.m, g->psi[p][mm.psi], F32, 4, px, g->ny, g->nz, px, mm.bx, mm.by)
                                : axis == 1 ? encode_map3(mm.m, g->psi[p][mm.psi], F32, 4, g->nx, d2, g->nz, g->pitch,
                                                          mm.bx, mm.by)
                                            : encode_map3(mm.m, g->psi[p][mm.psi], F32, 4, g->nx, g->ny, d2, g->pitch,
                                                          mm.bx, mm.by);
                if (!ok) return fail(g, FDTD_ECUDA, "cuTensorMapEncodeTiled failed for a CPML array");
            }
        }
    }
    g->ncx = (g->nx + TX - 1) / TX;
    g->ncy = (g->ny + TY - 1) / TY;
    const int cols = g->ncx * g->ncy, d = g->d;
    int dev = 0, sms = 0, smem_per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e != cudaSuccess) return cuda_fail(g, e, "device query");
    int max_smem = 0;
    for (int l = 0; l < 2; ++l) {
        auto &L = g->lc[l];
        L = {};
        L.work = g->work_d + 2 * l;
        if (l == 0) {            // planes between the z layers (all planes without a CPML)
            L.zlo = d;
            L.zhi = g->nz - d;
            L.kz = std::min(L.zhi - L.zlo, g->block > 0 ? g->block : 16);
            L.zxy = 0;
        } else {                 // the two z layers, one block each
            if (d == 0) break;
            L.zlo = 0;
            L.zhi = d;
            L.zlo2 = g->nz - d;
            L.zhi2 = g->nz;
            L.kz = d;
            L.zxy = 1;
        }
        const int nzb = (L.zhi - L.zlo + L.kz - 1) / L.kz + (L.zhi2 - L.zlo2 + L.kz - 1) / L.kz;
        L.nitems = cols * nzb;
        fdtd::step_region(g->pg, L.zxy, &L.region, &L.ox, &L.oy);
        // three H slots (two planes of lookahead) unless that costs the
        // second resident CTA per SM
        L.nh = 3;
        if (2 * (fdtd::step_smem_bytes(g->n_classes, d, L.region, 3) + 1024) > smem_per_sm &&
            2 * (fdtd::step_smem_bytes(g->n_classes, d, L.region, 2) + 1024) <= smem_per_sm)
            L.nh = 2;
        max_smem = std::max(max_smem, fdtd::step_smem_bytes(g->n_classes, d, L.region, L.nh));
        g->n_launch = l + 1;
    }
    const bool wide = grid_is_wide(g);
    for (int nh = 2; nh <= 3 && e == cudaSuccess; ++nh) e = ensure_smem(fdtd::step_kernel_ptr(nh, false, wide), max_smem);
    if (e != cudaSuccess) return cuda_fail(g, e, "step kernel setup");
    for (int l = 0; l < g->n_launch; ++l) {
        auto &L = g->lc[l];
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fdtd::step_kernel_ptr(L.nh, false, wide), fdtd::step_threads(),
                                                          fdtd::step_smem_bytes(g->n_classes, d, L.region, L.nh));
        if (e != cudaSuccess) return cuda_fail(g, e, "step kernel occupancy");
        if (occ < 1) return fail(g, FDTD_ECUDA, "step kernel does not fit on an SM");
        L.grid = std::max(1, std::min(sms * occ, L.nitems));
    }
    g->sms = sms;
    return FDTD_OK;
}

// the watchdog's check of the current state, queued on s
cudaError_t enqueue_watch(fdtd_grid *g, cudaStream_t s)
{
    fdtd::FieldPtrs f{};
    for (int c = 0; c < 6; ++c) f.p[c] = g->F[g->parity][c];
    return fdtd::launch_finite_check(f, (long long)g->plane * g->nz, g->div_d, 4 * std::max(g->sms, 1), s);
}

// Capture the graphs of 2, 4, 8, 16 and 32 steps from parity 0 (all at the
// first call that needs one, so no later call pays a capture)
int capture_graphs(fdtd_grid *g)
{
    nvtxRangePushA("fdtd_step graph capture");
    cudaError_t e = cudaSuccess;
    if (!g->cap_stream) e = cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking);
    for (int k = 1; k <= 5 && e == cudaSuccess; ++k) {
        const int len = 1 << k;
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            for (int t = 0; t < len && e == cudaSuccess; ++t) e = enqueue_step(g, t & 1, g->cap_stream, t, t == len - 1);
            cudaError_t e2 = cudaStreamEndCapture(g->cap_stream, &graph);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&g->graph[k], graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) g->graph[k] = nullptr;
    }
    nvtxRangePop();
    return e == cudaSuccess ? FDTD_OK : cuda_fail(g, e, "graph capture");
}

// n steps: graph replays of 32, 16, 8, 4 or 2 steps (from parity 0, the
// largest that fits) while the parity allows, direct launches otherwise; the
// watchdog's check after every replay or step that crosses a multiple of its
// period
int step_queue(fdtd_grid *g, int n)
{
    while (n > 0) {
        const long before = g->step;
        if (g->parity == 0 && n >= 2) {
            int k = 1;
            while (k < 5 && (2 << k) <= n) ++k;          // largest 2^k <= min(n, 32)
            const int len = 1 << k;
            if (!g->graph[k])
                if (int rc = capture_graphs(g)) return rc;
            cudaError_t e = cudaGraphLaunch(g->graph[k], g->stream);
            if (e != cudaSuccess) return cuda_fail(g, e, "graph launch");
            n -= len;
            g->step += len;
        } else {
            cudaError_t e = enqueue_step(g, g->parity, g->stream);
            if (e != cudaSuccess) return cuda_fail(g, e, "step launch");
            g->parity ^= 1;
            n -= 1;
            g->step += 1;
        }
        if (g->watch > 0 && g->step / g->watch != before / g->watch) {
            cudaError_t e = enqueue_watch(g, g->stream);
            if (e != cudaSuccess) return cuda_fail(g, e, "watchdog launch");
        }
    }
    return FDTD_OK;
}

int check_open(fdtd_grid *g, bool want_finalized)
{
    if (!g) return FDTD_EINVAL;
    if (g->finalized != want_finalized)
        return fail(g, FDTD_ESTATE, want_finalized ? "grid not finalized" : "grid already finalized");
    return FDTD_OK;
}

}  // namespace

namespace fdtd {

int set_error(fdtd_grid *g, int code, const char *msg) { return fail(g, code, msg); }

// n steps by direct launches, with the step kernel's work counters (two per
// launch, scratch[0 .. 2 * launches)) and its error flag (the last int,
// scratch[scratch_ints - 1], the same slot for every grid) taken from
// `scratch` instead of the grid's arena; nothing is allocated.  The counters
// are cleared on the grid's stream first; the error flag is left for
// fdtd_synchronize(), which reads and clears it.
int step_with_scratch(fdtd_grid *g, int n, int *scratch, int scratch_ints)
{
    if (int rc = check_open(g, true)) return rc;
    if (n < 0) return fail(g, FDTD_EINVAL, "negative step count");
    if (2 * g->n_launch > scratch_ints - 1)
        return fail(g, FDTD_EINVAL, "the step needs more scratch than the static array holds");
    cudaError_t e = cudaMemsetAsync(scratch, 0, 2 * g->n_launch * sizeof(int), g->stream);
    if (e != cudaSuccess) return cuda_fail(g, e, "scratch clear");
    g->noalloc_err = scratch + (scratch_ints - 1);
    for (; n > 0; --n) {
        if (!g->osegs.empty()) e = launch_wire_gather(edge_args(g, g->parity), g->stream);
        for (int l = 0; l < g->n_launch && e == cudaSuccess; ++l)
            e = launch_step(single_args(g, g->parity, l), grid_launch(g, g->parity, l, scratch + 2 * l, g->noalloc_err),
                            g->lc[l].grid, g->stream);
        if (e == cudaSuccess && g->npoles && !g->osegs.empty())
            e = launch_wire_finish(edge_args(g, g->parity), g->stream);
        if (e == cudaSuccess && g->npoles) e = launch_debye(debye_args(g, g->parity), g->stream);
        if (e == cudaSuccess && has_edge_work(g))
            e = launch_edges(edge_args(g, g->parity), g->stream);
        if (e != cudaSuccess) return cuda_fail(g, e, "step launch");
        g->parity ^= 1;
        g->step += 1;
    }
    return FDTD_OK;
}

}  // namespace fdtd

extern "C" {

int fdtd_create_grid(int nx, int ny, int nz, double dx, double courant, const fdtd_cpml *cpml,
                     void *cuda_stream, fdtd_grid **out)
{
    if (!out) return FDTD_EINVAL;
    *out = nullptr;
    if (nx < 2 || ny < 2 || nz < 2 || !(dx > 0) || !std::isfinite(dx)) return FDTD_EINVAL;
    if (!(courant > 0) || courant > 1.0) return FDTD_ECOURANT;
    int d = cpml ? cpml->cells : 0;
    if (d < 0) return FDTD_EINVAL;
    if (d > 0 && (nx < 2 * d + 2 || ny < 2 * d + 2 || nz < 2 * d + 2)) return FDTD_EINVAL;
    // the step kernel indexes the compact CPML auxiliaries with 32-bit integers
    if (d > 0) {
        const double pitch = (nx + 15) / 16 * 16, px = (2 * d + 3) / 4 * 4, d2 = 2.0 * d;
        if ((double)nz * ny * px >= 2147483647.0 || nz * d2 * pitch >= 2147483647.0 ||
            d2 * ny * pitch >= 2147483647.0)
            return FDTD_EINVAL;
    }
    if (d > 0 && (cpml->kappa_max < 1.0 || cpml->alpha_max < 0 || cpml->order < 0)) return FDTD_EINVAL;
    fdtd_grid *g = new (std::nothrow) fdtd_grid();
    if (!g) return FDTD_ENOMEM;
    g->nx = nx; g->ny = ny; g->nz = nz; g->dx = dx; g->courant = courant;
    g->dt = courant * dx / (kC0 * std::sqrt(3.0));
    g->d = d;
    if (d > 0) {
        g->cpml = *cpml;
        if (g->cpml.sigma_max <= 0)
            g->cpml.sigma_max = 0.8 * (g->cpml.order + 1.0) / (std::sqrt(kMu0 / kEps0) * dx);
    }
    g->stream = (cudaStream_t)cuda_stream;
    g->pitch = (nx + 15) / 16 * 16;   // 16-byte rows even for the class bytes (TMA strides)
    g->plane = (long long)g->pitch * ny;
    g->mat.assign((size_t)nx * ny * nz, 0);
    g->table.push_back(fdtd_material{1.0, 0.0, 1.0});
    *out = g;
    return FDTD_OK;
}

int fdtd_set_materials(fdtd_grid *g, const uint8_t *cell_material, const fdtd_material *table,
                       int n_materials)
{
    if (int rc = check_open(g, false)) return rc;
    if (!cell_material || !table || n_materials < 1 || n_materials > 256)
        return fail(g, FDTD_EINVAL, "bad material arguments");
    for (int m = 0; m < n_materials; ++m)
        if (!(table[m].eps_r > 0) || !(table[m].sigma >= 0) || !(table[m].mu_r > 0))
            return fail(g, FDTD_EINVAL, "material " + std::to_string(m) + " out of range");
    const size_t nc = g->mat.size();
    for (size_t c = 0; c < nc; ++c)
        if (cell_material[c] >= n_materials) return fail(g, FDTD_EINVAL, "material index out of range");
    std::memcpy(g->mat.data(), cell_material, nc);
    g->table.assign(table, table + n_materials);
    return FDTD_OK;
}

int fdtd_set_debye(fdtd_grid *g, int material, int n_poles, const double *delta_eps, const double *tau)
{
    if (int rc = check_open(g, false)) return rc;
    if (material < 0 || material > 255 || n_poles < 0 || n_poles > fdtd::kMaxPoles ||
        (n_poles > 0 && (!delta_eps || !tau)))
        return fail(g, FDTD_EINVAL, "bad Debye arguments");
    for (int p = 0; p < n_poles; ++p)
        if (!(delta_eps[p] >= 0) || !(tau[p] > 0))
            return fail(g, FDTD_EINVAL, "Debye pole " + std::to_string(p) + " out of range");
    auto &P = g->poles[material];
    for (int p = 0; p < fdtd::kMaxPoles; ++p) {
        P[p] = p < n_poles ? delta_eps[p] : 0.0;
        P[fdtd::kMaxPoles + p] = p < n_poles ? tau[p] : 1.0;
    }
    return FDTD_OK;
}

int fdtd_add_wire(fdtd_grid *g, int i0, int j0, int k0, int i1, int j1, int k1, double radius,
                  int *wire_id)
{
    if (int rc = check_open(g, false)) return rc;
    Wire w{};
    const int lo[3] = {i0, j0, k0}, hi[3] = {i1, j1, k1}, n[3] = {g->nx, g->ny, g->nz};
    int axis = -1;
    for (int u = 0; u < 3; ++u)
        if (hi[u] != lo[u]) {
            if (axis >= 0 || hi[u] < lo[u]) return fail(g, FDTD_EINVAL, "wire must run along +x, +y or +z");
            axis = u;
        }
    if (axis < 0) return fail(g, FDTD_EINVAL, "wire has zero length");
    for (int u = 0; u < 3; ++u) {
        if (u == axis) { if (lo[u] < 0 || hi[u] > n[u]) return fail(g, FDTD_EINVAL, "wire outside the grid"); }
        else if (lo[u] < 1 || lo[u] > n[u] - 1) return fail(g, FDTD_EINVAL, "wire must lie inside the walls");
    }
    if (!(radius > 0) || radius > kR0 * g->dx * (1.0 + 1e-12))
        return fail(g, FDTD_EINVAL, "wire radius must be in (0, 0.23 dx]");
    w.axis = axis;
    std::memcpy(w.p, lo, sizeof w.p);
    w.n = hi[axis] - lo[axis];
    w.radius = radius;
    g->wires.push_back(w);
    if (wire_id) *wire_id = (int)g->wires.size() - 1;
    return FDTD_OK;
}

int fdtd_add_wire_path(fdtd_grid *g, int i0, int j0, int k0, int i1, int j1, int k1, double radius,
                       int *n_segments)
{
    if (int rc = check_open(g, false)) return rc;
    const int a[3] = {i0, j0, k0}, b[3] = {i1, j1, k1};
    int d[3], len = 0;
    for (int u = 0; u < 3; ++u) {
        d[u] = std::abs(b[u] - a[u]);
        len += d[u];
    }
    if (len == 0) return fail(g, FDTD_EINVAL, "wire has zero length");
    // unit steps: along the axis least advanced towards b, ties to the lowest
    std::vector<int> steps;
    int c[3] = {i0, j0, k0};
    for (int s = 0; s < len; ++s) {
        int best = -1;
        double bp = 2.0;
        for (int u = 0; u < 3; ++u) {
            if (c[u] == b[u]) continue;
            const double prog = (double)std::abs(c[u] - a[u]) / d[u];
            if (prog < bp) { bp = prog; best = u; }
        }
        steps.push_back(best);
        c[best] += b[best] > a[best] ? 1 : -1;
    }
    // runs along one axis become wires (from the lower node)
    const size_t before = g->wires.size();
    int at[3] = {i0, j0, k0}, added = 0;
    for (size_t s = 0; s < steps.size();) {
        const int u = steps[s];
        size_t e = s;
        while (e < steps.size() && steps[e] == u) ++e;
        int p0[3] = {at[0], at[1], at[2]};
        at[u] += (b[u] > a[u] ? 1 : -1) * (int)(e - s);
        int p1[3] = {at[0], at[1], at[2]};
        if (p1[u] < p0[u]) std::swap(p0[u], p1[u]);
        if (int rc = fdtd_add_wire(g, p0[0], p0[1], p0[2], p1[0], p1[1], p1[2], radius, nullptr)) {
            g->wires.resize(before);           // nothing of the path stays
            return rc;
        }
        ++added;
        s = e;
    }
    if (n_segments) *n_segments = added;
    return FDTD_OK;
}

int fdtd_add_source(fdtd_grid *g, int i, int j, int k, int axis, double r_internal,
                    const double *current, int n_samples, int *source_id)
{
    if (int rc = check_open(g, false)) return rc;
    if (axis < 0 || axis > 2 || n_samples < 0 || (n_samples > 0 && !current))
        return fail(g, FDTD_EINVAL, "bad source arguments");
    if (!(r_internal >= 0)) return fail(g, FDTD_EINVAL, "negative internal resistance");
    Source s;
    s.axis = axis;
    s.p[0] = i; s.p[1] = j; s.p[2] = k;
    if (!e_updated(g, axis, s.p)) return fail(g, FDTD_EINVAL, "source edge on a wall or outside the grid");
    s.cur.resize(n_samples);
    for (int t = 0; t < n_samples; ++t) s.cur[t] = (float)current[t];
    if (r_internal > 0) g->lumps.push_back(Lump{axis, {i, j, k}, 0.0, 1.0 / (r_internal * g->dx)});
    g->srcs.push_back(std::move(s));
    if (source_id) *source_id = (int)g->srcs.size() - 1;
    return FDTD_OK;
}

int fdtd_add_voltage_source(fdtd_grid *g, int i, int j, int k, int axis, double r_internal, const double *voltage,
                            int n_samples, int *source_id)
{
    if (int rc = check_open(g, false)) return rc;
    if (axis < 0 || axis > 2 || n_samples < 0 || (n_samples > 0 && !voltage) || !(r_internal >= 0))
        return fail(g, FDTD_EINVAL, "bad voltage source arguments");
    Source s;
    s.axis = axis;
    s.p[0] = i; s.p[1] = j; s.p[2] = k;
    if (!e_updated(g, axis, s.p)) return fail(g, FDTD_EINVAL, "source edge on a wall or outside the grid");
    s.cur.resize(n_samples);
    if (r_internal == 0) {              // ideal: the edge's E is set to -V / dx
        s.hard = 1;
        for (int t = 0; t < n_samples; ++t) s.cur[t] = (float)voltage[t];
    } else {                            // Norton equivalent: V / R in parallel with R
        for (int t = 0; t < n_samples; ++t) s.cur[t] = (float)(voltage[t] / r_internal);
        g->lumps.push_back(Lump{axis, {i, j, k}, 0.0, 1.0 / (r_internal * g->dx)});
    }
    g->srcs.push_back(std::move(s));
    if (source_id) *source_id = (int)g->srcs.size() - 1;
    return FDTD_OK;
}

int fdtd_add_lumped(fdtd_grid *g, int i, int j, int k, int axis, double resistance, double capacitance,
                    int *element_id)
{
    if (int rc = check_open(g, false)) return rc;
    if (axis < 0 || axis > 2 || !(resistance >= 0) || !(capacitance >= 0) || (resistance == 0 && capacitance == 0))
        return fail(g, FDTD_EINVAL, "bad lumped element arguments");
    const int p[3] = {i, j, k};
    if (!e_updated(g, axis, p)) return fail(g, FDTD_EINVAL, "lumped element edge on a wall or outside the grid");
    g->lumps.push_back(Lump{axis, {i, j, k}, capacitance / g->dx, resistance > 0 ? 1.0 / (resistance * g->dx) : 0.0});
    if (element_id) *element_id = (int)g->lumps.size() - 1;
    return FDTD_OK;
}

int fdtd_add_probe(fdtd_grid *g, int kind, int i, int j, int k, int axis, int n_edges, int *probe_id)
{
    if (int rc = check_open(g, false)) return rc;
    if (kind < 0 || kind > 3 || axis < 0 || axis > 2) return fail(g, FDTD_EINVAL, "bad probe kind or axis");
    const int p[3] = {i, j, k}, n[3] = {g->nx, g->ny, g->nz};
    for (int u = 0; u < 3; ++u)
        if (p[u] < 0 || p[u] >= n[u]) return fail(g, FDTD_EINVAL, "probe outside the grid");
    if (kind == FDTD_PROBE_V) {
        if (n_edges < 1 || p[axis] + n_edges > n[axis]) return fail(g, FDTD_EINVAL, "voltage path outside the grid");
    } else {
        n_edges = 1;
    }
    if (kind == FDTD_PROBE_I)
        for (int u = 0; u < 3; ++u)
            if (u != axis && p[u] < 1) return fail(g, FDTD_EINVAL, "current loop needs transverse index >= 1");
    g->probes.push_back(fdtd::ProbeDesc{kind, axis, i, j, k, n_edges});
    if (probe_id) *probe_id = (int)g->probes.size() - 1;
    return FDTD_OK;
}

int fdtd_add_oblique_wire(fdtd_grid *g, double x0, double y0, double z0, double x1, double y1, double z1,
                          double radius, int *wire_id)
{
    if (int rc = check_open(g, false)) return rc;
    const double A[3] = {x0, y0, z0}, B[3] = {x1, y1, z1};
    const int n[3] = {g->nx, g->ny, g->nz};
    double len2 = 0.0;
    for (int u = 0; u < 3; ++u) {
        if (!(A[u] >= 0.0 && A[u] <= n[u] && B[u] >= 0.0 && B[u] <= n[u]))
            return fail(g, FDTD_EINVAL, "oblique wire outside the grid");
        len2 += (B[u] - A[u]) * (B[u] - A[u]);
    }
    const double len = std::sqrt(len2);
    if (!(len >= 0.5)) return fail(g, FDTD_EINVAL, "oblique wire shorter than half a cell");
    if (!(radius > 0.0) || radius > 0.1 * g->dx) return fail(g, FDTD_EINVAL, "oblique wire radius outside (0, 0.1 dx]");
    const int N = (int)std::max(1L, std::lround(len));
    auto node_at = [&](const double p[3]) {
        for (size_t m = 0; m < g->onodes.size(); ++m)
            if (std::fabs(g->onodes[m].p[0] - p[0]) < 1e-9 && std::fabs(g->onodes[m].p[1] - p[1]) < 1e-9 &&
                std::fabs(g->onodes[m].p[2] - p[2]) < 1e-9)
                return (int)m;
        return -1;
    };
    auto new_node = [&](const double p[3]) {
        ONodeH nd{{p[0], p[1], p[2]}, 0};
        for (int u = 0; u < 3; ++u) nd.grounded |= (p[u] == 0.0 || p[u] == (double)n[u]);
        g->onodes.push_back(nd);
        return (int)g->onodes.size() - 1;
    };
    g->owires.push_back(OWireH{(int)g->osegs.size(), N});
    int prev = node_at(A);
    if (prev < 0) prev = new_node(A);
    for (int sg = 0; sg < N; ++sg) {
        double P[3], c[3], t[3];
        for (int u = 0; u < 3; ++u) {
            P[u] = sg == N - 1 ? B[u] : A[u] + (B[u] - A[u]) * (double)(sg + 1) / N;
            c[u] = A[u] + (B[u] - A[u]) * (sg + 0.5) / N;
            t[u] = (B[u] - A[u]) / len;
        }
        int next = sg == N - 1 ? node_at(B) : -1;
        if (next < 0) next = new_node(P);
        OSegH seg;
        seg.a = prev;
        seg.b = next;
        seg.dl = len * g->dx / N;
        seg.lam = std::log(lattice_radius(g->dx, c, t) / radius);
        for (int u = 0; u < 3; ++u) { seg.c[u] = c[u]; seg.t[u] = t[u]; }
        for (int u = 0; u < 3; ++u) seg.cell[u] = std::min((int)std::floor(c[u]), n[u] - 1);
        const ONodeH pa = g->onodes[prev], pb = g->onodes[next];
        seg.edges = path_edges(g, pa.p, pb.p);
        g->osegs.push_back(std::move(seg));
        prev = next;
    }
    if (wire_id) *wire_id = (int)g->owires.size() - 1;
    return FDTD_OK;
}

int fdtd_add_wire_voltage_source(fdtd_grid *g, int wire_id, int segment, double r_internal, const double *voltage,
                                 int n, int *source_id)
{
    if (int rc = check_open(g, false)) return rc;
    if (wire_id < 0 || wire_id >= (int)g->owires.size() || segment < 0 || segment >= g->owires[wire_id].nseg)
        return fail(g, FDTD_EINVAL, "no such oblique-wire segment");
    if (n < 0 || (n > 0 && !voltage)) return fail(g, FDTD_EINVAL, "bad voltage samples");
    if (!(r_internal >= 0.0) || !std::isfinite(r_internal)) return fail(g, FDTD_EINVAL, "bad internal resistance");
    OSrcH sr{g->owires[wire_id].seg0 + segment, std::vector<float>(voltage, voltage + n), r_internal};
    g->osrcs.push_back(std::move(sr));
    if (source_id) *source_id = (int)g->osrcs.size() - 1;
    return FDTD_OK;
}

int fdtd_add_wire_probe(fdtd_grid *g, int wire_id, int segment, int *probe_id)
{
    if (int rc = check_open(g, false)) return rc;
    if (wire_id < 0 || wire_id >= (int)g->owires.size() || segment < 0 || segment >= g->owires[wire_id].nseg)
        return fail(g, FDTD_EINVAL, "no such oblique-wire segment");
    g->probes.push_back(fdtd::ProbeDesc{FDTD_PROBE_WIRE, 0, g->owires[wire_id].seg0 + segment, 0, 0, 1});
    if (probe_id) *probe_id = (int)g->probes.size() - 1;
    return FDTD_OK;
}

int fdtd_add_wire_node_probe(fdtd_grid *g, double x, double y, double z, int *probe_id)
{
    if (int rc = check_open(g, false)) return rc;
    for (size_t m = 0; m < g->onodes.size(); ++m)
        if (std::fabs(g->onodes[m].p[0] - x) < 1e-9 && std::fabs(g->onodes[m].p[1] - y) < 1e-9 &&
            std::fabs(g->onodes[m].p[2] - z) < 1e-9) {
            g->probes.push_back(fdtd::ProbeDesc{FDTD_PROBE_WIRE_V, 0, (int)m, 0, 0, 1});
            if (probe_id) *probe_id = (int)g->probes.size() - 1;
            return FDTD_OK;
        }
    return fail(g, FDTD_EINVAL, "no oblique-wire node at that point");
}

int fdtd_wire_courant_limit(const fdtd_grid *g, double *courant)
{
    if (!g || !courant) return FDTD_EINVAL;
    *courant = wire_courant_limit(g);
    return FDTD_OK;
}

int fdtd_wire_counts(const fdtd_grid *g, int *n_segments, int *n_nodes)
{
    if (!g || !n_segments || !n_nodes) return FDTD_EINVAL;
    *n_segments = (int)g->osegs.size();
    *n_nodes = (int)g->onodes.size();
    return FDTD_OK;
}

int fdtd_get_wire_state(fdtd_grid *g, float *I, float *Q)
{
    if (int rc = check_open(g, true)) return rc;
    if ((!I && !g->osegs.empty()) || (!Q && !g->onodes.empty())) return fail(g, FDTD_EINVAL, "null buffer");
    cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e == cudaSuccess && !g->osegs.empty())
        e = cudaMemcpy(I, g->oI_d, g->osegs.size() * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && !g->onodes.empty())
        e = cudaMemcpy(Q, g->oQ_d, g->onodes.size() * sizeof(float), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? FDTD_OK : cuda_fail(g, e, "wire state read");
}

int fdtd_set_wire_state(fdtd_grid *g, const float *I, const float *Q)
{
    if (int rc = check_open(g, true)) return rc;
    if ((!I && !g->osegs.empty()) || (!Q && !g->onodes.empty())) return fail(g, FDTD_EINVAL, "null buffer");
    std::vector<float> q(Q, Q + g->onodes.size()), v(g->onodes.size()), p(4 * g->onodes.size(), 0.f);
    std::vector<fdtd::ONode> nd(g->onodes.size());
    cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e == cudaSuccess && !nd.empty())
        e = cudaMemcpy(nd.data(), g->onode_d, nd.size() * sizeof(fdtd::ONode), cudaMemcpyDeviceToHost);
    for (size_t m = 0; m < q.size(); ++m) {
        if (g->onodes[m].grounded) q[m] = 0.f;       // grounded nodes hold no charge
        v[m] = nd.empty() ? 0.f : nd[m].K * q[m] / nd[m].e0;   // polarisation-free
    }
    if (e == cudaSuccess && !g->osegs.empty())
        e = cudaMemcpy(g->oI_d, I, g->osegs.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !q.empty()) e = cudaMemcpy(g->oQ_d, q.data(), q.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !v.empty()) e = cudaMemcpy(g->oV_d, v.data(), v.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !p.empty()) e = cudaMemcpy(g->oP_d, p.data(), p.size() * sizeof(float), cudaMemcpyHostToDevice);
    return e == cudaSuccess ? FDTD_OK : cuda_fail(g, e, "wire state write");
}

int fdtd_set_block(fdtd_grid *g, int planes)
{
    if (int rc = check_open(g, false)) return rc;
    if (planes < 0 || planes > 256) return fail(g, FDTD_EINVAL, "planes per work item outside 0..256");
    g->block = planes;
    return FDTD_OK;
}

int fdtd_bounds_report(fdtd_grid *g, int *site, int *count)
{
    if (int rc = check_open(g, true)) return rc;
    if (int rc = fdtd_synchronize(g)) return rc;
    int v[2] = {0, 0};
    cudaError_t e = cudaMemcpy(v, g->work_d + 6, sizeof v, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(g, e, "bounds record read");
    if (site) *site = v[0];
    if (count) *count = v[1];
#ifdef FDTD_BOUNDS
    return FDTD_OK;
#else
    return 1;                    // not the bounds-checked build: nothing was checked
#endif
}

int fdtd_set_watchdog(fdtd_grid *g, int every)
{
    if (!g) return FDTD_EINVAL;
    if (every < 0) return fail(g, FDTD_EINVAL, "negative watchdog period");
    g->watch = every;
    return FDTD_OK;
}

int fdtd_arena_bytes(const fdtd_grid *g, int probe_capacity, size_t *bytes)
{
    if (!g || !bytes || probe_capacity < 0) return FDTD_EINVAL;
    *bytes = make_plan(g, probe_capacity).total;
    return FDTD_OK;
}

int fdtd_finalize(fdtd_grid *g, int probe_capacity, void *arena, size_t arena_bytes)
{
    if (int rc = check_open(g, false)) return rc;
    if (probe_capacity < 0) return fail(g, FDTD_EINVAL, "negative probe capacity");
    std::vector<uint8_t> cls, dcls;
    std::vector<float> table, dtable;
    std::vector<double> src_cb;
    std::vector<std::array<double, 3 * fdtd::kMaxPoles>> src_debye;
    if (int rc = build_classes(g, cls, table, src_cb, dcls, dtable, src_debye)) return rc;
    // an oblique-wire node on the node line of an axis-aligned wire joins that
    // conductor: grounded to it like a node on the wall, its charge handed to
    // the grid, where the PEC line carries it
    for (ONodeH &nd : g->onodes)
        for (const Wire &w : g->wires) {
            bool on = true;
            for (int u = 0; u < 3; ++u)
                on = on && (u == w.axis ? nd.p[u] >= w.p[u] - 1e-9 && nd.p[u] <= w.p[u] + w.n + 1e-9
                                        : std::fabs(nd.p[u] - w.p[u]) <= 1e-9);
            if (on) nd.grounded = 1;
        }
    if (!g->osegs.empty() && g->courant > wire_courant_limit(g)) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "the oblique wires need courant <= %.4f (thinner wires or a smaller step)",
                      wire_courant_limit(g));
        return fail(g, FDTD_ECOURANT, msg);
    }

    const Plan p = make_plan(g, probe_capacity);
    if (arena) {
        if (arena_bytes < p.total) return fail(g, FDTD_ENOMEM, "arena smaller than fdtd_arena_bytes()");
        if ((uintptr_t)arena % 256) return fail(g, FDTD_EINVAL, "arena must be 256-byte aligned");
        g->arena = arena;
        g->own_arena = false;
    } else {
        cudaError_t e = cudaMalloc(&g->arena, p.total);
        if (e != cudaSuccess) { g->arena = nullptr; return fail(g, FDTD_ENOMEM, "cudaMalloc of the arena failed"); }
        g->own_arena = true;
    }
    g->arena_bytes = p.total;
    char *base = (char *)g->arena;
    const size_t cells = (size_t)g->plane * g->nz;
    for (int b = 0; b < 2; ++b)
        for (int c = 0; c < 6; ++c) g->F[b][c] = (float *)(base + p.field) + (size_t)(b * 6 + c) * cells;
    g->cls = (uint8_t *)(base + p.cls);
    g->table_d = (float *)(base + p.table);
    for (int u = 0; u < 3; ++u) g->prof[u] = (float *)(base + p.prof[u]);
    for (int q = 0; q < fdtd::PSI_COUNT; ++q) {
        const size_t n = psi_elems(g, q);
        g->psi[0][q] = n ? (float *)(base + p.psi[q]) : nullptr;
        g->psi[1][q] = n ? (float *)(base + p.psi[q]) + n : nullptr;
    }
    g->src_d = (fdtd::SourceDesc *)(base + p.src);
    g->samples_d = (float *)(base + p.samples);
    g->probes_d = (fdtd::ProbeDesc *)(base + p.probes);
    g->probe_out = (float *)(base + p.out);
    g->step_d = (long long *)(base + p.step);
    g->work_d = (int *)(base + p.work);
    g->err_d = g->work_d + 4;
    g->div_d = g->work_d + 5;
    g->slot_d = (fdtd::DomainSlot *)(base + p.slot);
    g->item_start_d = (int *)(base + p.items);
    g->isrc_d = (int2 *)(base + p.isrc);
    g->order_d = (int *)(base + p.order);
    g->J = (float *)(base + p.J);
    g->dcls_d = (uint8_t *)(base + p.dcls);
    g->dtable_d = (float *)(base + p.dtable);
    g->oseg_d = (fdtd::OSeg *)(base + p.oseg);
    g->ochunk_d = (int *)(base + p.ochunk);
    g->oedge_d = (fdtd::OEdge *)(base + p.oedge);
    g->oscat_d = (fdtd::OScat *)(base + p.oscat);
    g->oterm_d = (fdtd::OTerm *)(base + p.oterm);
    g->onode_d = (fdtd::ONode *)(base + p.onode);
    g->oadj_d = (int *)(base + p.oadj);
    g->oI_d = (float *)(base + p.oI);
    g->oQ_d = (float *)(base + p.oQ);
    g->oV_d = (float *)(base + p.oV);
    g->oP_d = (float *)(base + p.oP);
    g->osrc_d = (fdtd::OSrc *)(base + p.osrc);
    g->osamp_d = (float *)(base + p.osamp);
    g->capacity = probe_capacity;


    cudaStream_t s = g->stream;
    cudaError_t e = cudaMemsetAsync(g->arena, 0, p.total, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->cls, cls.data(), cls.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->table_d, table.data(), table.size() * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && g->npoles) {
        const size_t box = (size_t)(g->dz1 - g->dz0) * g->plane;
        e = cudaMemcpyAsync(g->dcls_d, dcls.data() + (size_t)g->dz0 * g->plane, box, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g->dtable_d, dtable.data(), dtable.size() * sizeof(float), cudaMemcpyHostToDevice, s);
    }
    const int n[3] = {g->nx, g->ny, g->nz};
    for (int u = 0; u < 3 && e == cudaSuccess; ++u) {
        std::vector<float> pr = cpml_profile(g, n[u]);
        e = cudaMemcpyAsync(g->prof[u], pr.data(), pr.size() * sizeof(float), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // pr goes out of scope
    }
    std::vector<fdtd::SourceDesc> sd;
    std::vector<float> samples;
    for (size_t q = 0; q < g->srcs.size(); ++q) {
        const Source &src = g->srcs[q];
        fdtd::SourceDesc d{};
        d.comp = src.axis;
        d.idx = (long long)src.p[2] * g->plane + (long long)src.p[1] * g->pitch + src.p[0];
        d.coef = (float)(-src_cb[q] / g->dx);
        d.n_samples = (int)src.cur.size();
        d.sample_off = (long long)samples.size();
        d.jidx = -1;
        bool disp = false;
        for (int p2 = 0; p2 < fdtd::kMaxPoles; ++p2) {
            d.be[p2] = (float)src_debye[q][3 * p2 + 2];
            disp |= d.be[p2] != 0.f;
        }
        if (disp) d.jidx = d.idx - (long long)g->dz0 * g->plane;
        d.hard = src.hard;
        d.vcoef = (float)(-1.0 / g->dx);
        samples.insert(samples.end(), src.cur.begin(), src.cur.end());
        sd.push_back(d);
    }
    if (e == cudaSuccess && !sd.empty())
        e = cudaMemcpyAsync(g->src_d, sd.data(), sd.size() * sizeof(sd[0]), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !samples.empty())
        e = cudaMemcpyAsync(g->samples_d, samples.data(), samples.size() * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !g->probes.empty())
        e = cudaMemcpyAsync(g->probes_d, g->probes.data(), g->probes.size() * sizeof(fdtd::ProbeDesc),
                            cudaMemcpyHostToDevice, s);
    WireDev wd;
    if (!g->osegs.empty()) wd = wire_device(g, cls, table);
    auto up = [&](void *dst, const void *src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
    };
    up(g->oseg_d, wd.seg.data(), wd.seg.size() * sizeof(fdtd::OSeg));
    up(g->ochunk_d, wd.chunk.data(), wd.chunk.size() * sizeof(int));
    g->n_ochunk = wd.chunk.empty() ? 0 : (int)wd.chunk.size() - 1;
    up(g->oedge_d, wd.edge.data(), wd.edge.size() * sizeof(fdtd::OEdge));
    up(g->oscat_d, wd.scat.data(), wd.scat.size() * sizeof(fdtd::OScat));
    up(g->oterm_d, wd.term.data(), wd.term.size() * sizeof(fdtd::OTerm));
    g->n_oscat = (int)wd.scat.size();
    up(g->onode_d, wd.node.data(), wd.node.size() * sizeof(fdtd::ONode));
    up(g->oadj_d, wd.adj.data(), wd.adj.size() * sizeof(int));
    up(g->osrc_d, wd.src.data(), wd.src.size() * sizeof(fdtd::OSrc));
    up(g->osamp_d, wd.samples.data(), wd.samples.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(g, e, "upload");
    if (int rc = setup_step_kernel(g)) return rc;
    {
        // column tiles of a z block, costliest first: those meeting an x and a
        // y layer, then one layer, then none (in tile order within each class)
        using namespace fdtd::geom;
        std::vector<int> order, cost;
        for (int cy = 0; cy < g->ncy; ++cy)
            for (int cx = 0; cx < g->ncx; ++cx) {
                const int x0 = cx * TX, y0 = cy * TY, d = g->d;
                const bool tx = d > 0 && (std::max(x0 - 1, 0) < d || std::min(x0 + TX, g->nx) - 1 >= g->nx - d);
                const bool ty = d > 0 && (std::max(y0 - 1, 0) < d || std::min(y0 + TY, g->ny) - 1 >= g->ny - d);
                order.push_back(cy * g->ncx + cx);
                cost.push_back((int)tx + (int)ty);
            }
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
        g->order_pos.assign(order.size(), 0);
        for (size_t q = 0; q < order.size(); ++q) g->order_pos[order[q]] = (int)q;
        e = cudaMemcpyAsync(g->order_d, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(g, e, "upload of the column order");
    }
    // current sources in the step kernel: each source's launch and work item
    g->fast = g->npoles == 0 && g->osegs.empty() && g->srcs.size() <= 32 && has_edge_work(g);
    for (const Source &src : g->srcs) g->fast = g->fast && !src.hard;
    if (g->fast && !g->srcs.empty()) {
        using namespace fdtd::geom;
        std::vector<int2> loc;
        for (const Source &src : g->srcs) {
            const int i = src.p[0], j = src.p[1], k = src.p[2];
            const int col = g->order_pos[(j / TY) * g->ncx + i / TX];
            int2 at{-1, -1};
            for (int l = 0; l < g->n_launch; ++l) {
                const auto &L = g->lc[l];
                const int nzb1 = (L.zhi - L.zlo + L.kz - 1) / L.kz;
                int zb = -1;
                if (k >= L.zlo && k < L.zhi) zb = (k - L.zlo) / L.kz;
                else if (k >= L.zlo2 && k < L.zhi2) zb = nzb1 + (k - L.zlo2) / L.kz;
                if (zb >= 0) at = int2{l, zb * g->ncx * g->ncy + col};
            }
            if (at.x < 0) return fail(g, FDTD_EINVAL, "a source edge lies outside every step launch");
            loc.push_back(at);
        }
        e = cudaMemcpyAsync(g->isrc_d, loc.data(), loc.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(g, e, "upload of the source locations");
    }
    if ((g->n_launch == 2 || !g->osegs.empty() || (g->fast && !g->probes.empty())) && !g->fk.side) {
        e = g->fk.init();
        if (e != cudaSuccess) return cuda_fail(g, e, "side stream");
    }
    // the grid as a one-domain step launch: descriptors and arguments per
    // launch and input parity, item ranges {0, items} per launch
    std::memset(&g->slot_h, 0, sizeof g->slot_h);
    int items[4] = {0, 0, 0, 0};
    for (int par = 0; par < 2; ++par) {
        g->slot_h.m[par] = g->maps[par];
        for (int l = 0; l < g->n_launch; ++l) g->slot_h.a[l][par] = step_args(g, par, l);
        g->edge_h[par] = edge_args(g, par);
    }
    for (int l = 0; l < g->n_launch; ++l) items[2 * l + 1] = g->lc[l].nitems;
    e = cudaMemcpyAsync(g->slot_d, &g->slot_h, sizeof g->slot_h, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->item_start_d, items, sizeof items, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(g, e, "upload of the launch descriptors");
    g->finalized = true;
    return FDTD_OK;
}

int fdtd_step(fdtd_grid *g, int n)
{
    if (int rc = check_open(g, true)) return rc;
    if (n < 0) return fail(g, FDTD_EINVAL, "negative step count");
    nvtxRangePushA("fdtd_step");
    const int rc = step_queue(g, n);
    nvtxRangePop();
    return rc;
}

int fdtd_synchronize(fdtd_grid *g)
{
    if (!g) return FDTD_EINVAL;
    cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_fail(g, e, "synchronize");
    if (g->finalized) {
        int flag = 0;
        e = cudaMemcpy(&flag, g->err_d, sizeof flag, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(g, e, "error flag read");
        if (flag) return fail(g, FDTD_ETIMEOUT, "a bounded wait in the step kernel gave up");
        e = cudaMemcpy(&flag, g->div_d, sizeof flag, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(g, e, "watchdog flag read");
        if (flag) {
            // reported once per detection; a later check finds it again if the fields still diverge
            e = cudaMemsetAsync(g->div_d, 0, sizeof flag, g->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
            if (e != cudaSuccess) return cuda_fail(g, e, "watchdog flag clear");
            return fail(g, FDTD_EDIVERGED, "the watchdog found a NaN or an infinity in the fields");
        }
        if (g->noalloc_err) {
            // the shared flag of fdtd_step_noalloc(): read and cleared on this
            // grid's stream (it never holds a work counter)
            e = cudaMemcpyAsync(&flag, g->noalloc_err, sizeof flag, cudaMemcpyDeviceToHost, g->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
            if (e != cudaSuccess) return cuda_fail(g, e, "error flag read");
            if (flag) {
                e = cudaMemsetAsync(g->noalloc_err, 0, sizeof flag, g->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
                if (e != cudaSuccess) return cuda_fail(g, e, "error flag clear");
                return fail(g, FDTD_ETIMEOUT, "a bounded wait in the step kernel gave up (fdtd_step_noalloc)");
            }
        }
    }
    return FDTD_OK;
}

int fdtd_read_probes(fdtd_grid *g, int probe_id, int first_step, int count, float *host_out)
{
    if (int rc = check_open(g, true)) return rc;
    if (probe_id < 0 || probe_id >= (int)g->probes.size() || first_step < 0 || count < 0 ||
        (long long)first_step + count > g->capacity || (count > 0 && !host_out))
        return fail(g, FDTD_EINVAL, "probe range outside the recorded window");
    if (int rc = fdtd_synchronize(g)) return rc;
    if (count == 0) return FDTD_OK;
    cudaError_t e = cudaMemcpy(host_out, g->probe_out + (size_t)probe_id * g->capacity + first_step,
                               (size_t)count * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(g, e, "probe copy");
    return FDTD_OK;
}

int fdtd_get_field(fdtd_grid *g, int component, float *host_out)
{
    if (int rc = check_open(g, true)) return rc;
    if (component < 0 || component > 5 || !host_out) return fail(g, FDTD_EINVAL, "bad component");
    if (int rc = fdtd_synchronize(g)) return rc;
    cudaError_t e = cudaMemcpy2D(host_out, (size_t)g->nx * sizeof(float), g->F[g->parity][component],
                                 (size_t)g->pitch * sizeof(float), (size_t)g->nx * sizeof(float),
                                 (size_t)g->ny * g->nz, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(g, e, "field copy");
    return FDTD_OK;
}

int fdtd_set_field(fdtd_grid *g, int component, const float *host_in)
{
    if (int rc = check_open(g, true)) return rc;
    if (component < 0 || component > 5 || !host_in) return fail(g, FDTD_EINVAL, "bad component");
    if (int rc = fdtd_synchronize(g)) return rc;
    cudaError_t e = cudaMemcpy2D(g->F[g->parity][component], (size_t)g->pitch * sizeof(float), host_in,
                                 (size_t)g->nx * sizeof(float), (size_t)g->nx * sizeof(float),
                                 (size_t)g->ny * g->nz, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(g, e, "field copy");
    return FDTD_OK;
}

int fdtd_field_device(fdtd_grid *g, int component, void **dptr, int *row_pitch, size_t *plane_pitch)
{
    if (int rc = check_open(g, true)) return rc;
    if (component < 0 || component > 5 || !dptr) return fail(g, FDTD_EINVAL, "bad component");
    *dptr = g->F[g->parity][component];
    if (row_pitch) *row_pitch = g->pitch;
    if (plane_pitch) *plane_pitch = (size_t)g->plane;
    return FDTD_OK;
}

double fdtd_get_dt(const fdtd_grid *g) { return g ? g->dt : 0.0; }
long fdtd_get_step(const fdtd_grid *g) { return g ? g->step : -1; }
int fdtd_num_classes(const fdtd_grid *g) { return g ? g->n_classes : -1; }
// ---- checkpoint / resume ----------------------------------------------------
namespace {
constexpr uint32_t kStateMagic = 0x53544446u;     // "FDTS"
constexpr uint32_t kStateVersion = 5;             // 5: the CPML auxiliaries in their compact layout
struct StateHeader {
    uint32_t magic, version;
    int32_t nx, ny, nz, d, n_probes, capacity, n_psi, npoles, dz0, dz1, n_oseg, n_onode;
    int64_t step;
};

size_t debye_elems(const fdtd_grid *g) { return 3 * (size_t)g->npoles * (size_t)(g->dz1 - g->dz0) * g->plane; }

size_t psi_state_elems(const fdtd_grid *g, int n_psi)
{
    size_t n = 0;
    for (int q = 0; q < n_psi; ++q) n += psi_elems(g, q);
    return n;
}

size_t state_bytes(const fdtd_grid *g, int n_psi)
{
    const size_t cells = (size_t)g->nx * g->ny * g->nz;
    return sizeof(StateHeader) + 6 * cells * sizeof(float) + psi_state_elems(g, n_psi) * sizeof(float) +
           g->probes.size() * (size_t)g->capacity * sizeof(float) + debye_elems(g) * sizeof(float) +
           (g->osegs.size() + 6 * g->onodes.size()) * sizeof(float);
}

// one cell-owned array between host (dense) and device (row pitch)
cudaError_t copy_array(fdtd_grid *g, float *dev, char *host, bool to_host)
{
    const size_t row = (size_t)g->nx * sizeof(float), dpitch = (size_t)g->pitch * sizeof(float);
    const size_t rows = (size_t)g->ny * g->nz;
    return to_host ? cudaMemcpy2D(host, row, dev, dpitch, row, rows, cudaMemcpyDeviceToHost)
                   : cudaMemcpy2D(dev, dpitch, host, row, row, rows, cudaMemcpyHostToDevice);
}
}  // namespace

int fdtd_save_state(fdtd_grid *g, void *host_buf, size_t *bytes)
{
    if (int rc = check_open(g, true)) return rc;
    if (!bytes) return fail(g, FDTD_EINVAL, "null size pointer");
    const int n_psi = g->d > 0 ? fdtd::PSI_COUNT : 0;
    const size_t need = state_bytes(g, n_psi);
    if (!host_buf) {
        *bytes = need;
        return FDTD_OK;
    }
    if (*bytes < need) {
        *bytes = need;
        return fail(g, FDTD_EINVAL, "state buffer too small");
    }
    if (int rc = fdtd_synchronize(g)) return rc;
    StateHeader h{kStateMagic, kStateVersion, g->nx, g->ny, g->nz, g->d, (int32_t)g->probes.size(), g->capacity,
                  n_psi, g->npoles, g->dz0, g->dz1, (int32_t)g->osegs.size(), (int32_t)g->onodes.size(),
                  (int64_t)g->step};
    char *p = static_cast<char *>(host_buf);
    std::memcpy(p, &h, sizeof h);
    p += sizeof h;
    const size_t arr = (size_t)g->nx * g->ny * g->nz * sizeof(float);
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < 6 && e == cudaSuccess; ++c, p += arr) e = copy_array(g, g->F[g->parity][c], p, true);
    // the auxiliaries as stored (compact layout, row padding included)
    for (int q = 0; q < n_psi && e == cudaSuccess; ++q) {
        const size_t nb = psi_elems(g, q) * sizeof(float);
        e = cudaMemcpy(p, g->psi[g->parity][q], nb, cudaMemcpyDeviceToHost);
        p += nb;
    }
    const size_t pbytes = g->probes.size() * (size_t)g->capacity * sizeof(float);
    if (e == cudaSuccess && pbytes) e = cudaMemcpy(p, g->probe_out, pbytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && debye_elems(g))
        e = cudaMemcpy(p + pbytes, g->J, debye_elems(g) * sizeof(float), cudaMemcpyDeviceToHost);
    char *pw = p + pbytes + debye_elems(g) * sizeof(float);
    if (e == cudaSuccess && !g->osegs.empty())
        e = cudaMemcpy(pw, g->oI_d, g->osegs.size() * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && !g->onodes.empty()) {
        char *pn = pw + g->osegs.size() * sizeof(float);
        const size_t nb = g->onodes.size() * sizeof(float);
        e = cudaMemcpy(pn, g->oQ_d, nb, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(pn + nb, g->oV_d, nb, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(pn + 2 * nb, g->oP_d, 4 * nb, cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) return cuda_fail(g, e, "state copy");
    *bytes = need;
    return FDTD_OK;
}

int fdtd_load_state(fdtd_grid *g, const void *host_buf, size_t bytes)
{
    if (int rc = check_open(g, true)) return rc;
    if (!host_buf || bytes < sizeof(StateHeader)) return fail(g, FDTD_EINVAL, "no state");
    StateHeader h;
    std::memcpy(&h, host_buf, sizeof h);
    const int n_psi = g->d > 0 ? fdtd::PSI_COUNT : 0;
    if (h.magic != kStateMagic || h.version != kStateVersion) return fail(g, FDTD_EINVAL, "not a saved state");
    if (h.nx != g->nx || h.ny != g->ny || h.nz != g->nz || h.d != g->d || h.n_probes != (int)g->probes.size() ||
        h.capacity != g->capacity || h.n_psi != n_psi || h.npoles != g->npoles || h.dz0 != g->dz0 ||
        h.dz1 != g->dz1 || h.n_oseg != (int)g->osegs.size() || h.n_onode != (int)g->onodes.size() || h.step < 0)
        return fail(g, FDTD_EINVAL, "state was saved from a differently shaped grid");
    if (bytes < state_bytes(g, n_psi)) return fail(g, FDTD_EINVAL, "state truncated");
    if (int rc = fdtd_synchronize(g)) return rc;
    const char *p = static_cast<const char *>(host_buf) + sizeof h;
    const size_t arr = (size_t)g->nx * g->ny * g->nz * sizeof(float);
    char *q = const_cast<char *>(p);
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < 6 && e == cudaSuccess; ++c, q += arr) e = copy_array(g, g->F[g->parity][c], q, false);
    for (int a = 0; a < n_psi && e == cudaSuccess; ++a) {
        const size_t nb = psi_elems(g, a) * sizeof(float);
        e = cudaMemcpy(g->psi[g->parity][a], q, nb, cudaMemcpyHostToDevice);
        q += nb;
    }
    const size_t pbytes = g->probes.size() * (size_t)g->capacity * sizeof(float);
    if (e == cudaSuccess && pbytes) e = cudaMemcpy(g->probe_out, q, pbytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && debye_elems(g))
        e = cudaMemcpy(g->J, q + pbytes, debye_elems(g) * sizeof(float), cudaMemcpyHostToDevice);
    const char *qw = q + pbytes + debye_elems(g) * sizeof(float);
    if (e == cudaSuccess && !g->osegs.empty())
        e = cudaMemcpy(g->oI_d, qw, g->osegs.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !g->onodes.empty()) {
        const char *qn = qw + g->osegs.size() * sizeof(float);
        const size_t nb = g->onodes.size() * sizeof(float);
        e = cudaMemcpy(g->oQ_d, qn, nb, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(g->oV_d, qn + nb, nb, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(g->oP_d, qn + 2 * nb, 4 * nb, cudaMemcpyHostToDevice);
    }
    const long long step = h.step;
    if (e == cudaSuccess) e = cudaMemcpy(g->step_d, &step, sizeof step, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(g, e, "state copy");
    g->step = (long)h.step;
    return FDTD_OK;
}

const char *fdtd_last_error(const fdtd_grid *g) { return g ? g->err.c_str() : "null grid"; }

void fdtd_destroy(fdtd_grid *g)
{
    if (!g) return;
    if (g->finalized) cudaStreamSynchronize(g->stream);
    for (cudaGraphExec_t gr : g->graph)
        if (gr) cudaGraphExecDestroy(gr);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    g->fk.destroy();
    if (g->own_arena && g->arena) cudaFree(g->arena);
    delete g;
}

}  // extern "C"

// ---- batched engine ----------------------------------------------------
// Many finalized grids advanced together: each step is one persistent
// launch of the step kernel over the work items of every domain (and one
// over their z-layer planes when they have a CPML), then one source / probe
// launch with a CTA per domain.  fdtd_batch_step replays a captured graph.
struct fdtd_batch {
    std::vector<fdtd_grid *> grids;
    cudaStream_t stream = nullptr;
    void *mem = nullptr;
    fdtd::DomainSlot *doms = nullptr;
    int *item_start[2] = {};
    fdtd::EdgeArgs *edges = nullptr;
    int *work = nullptr;            // [2 per launch]
    int *errf = nullptr;
    int4 *img = nullptr;            // domains' staging images (fdtd_internal.h)
    int2 *img_ref = nullptr;        // [domain][launch][parity] {offset, length} in int4
    int nitems[2] = {}, grid[2] = {}, region[2] = {}, nh[2] = {};
    int max_classes = 0, max_d = 0, n_launch = 0;
    bool has_edges = false;
    bool has_wires = false;         // some domain has oblique wires
    cudaStream_t cap = nullptr;
    Fork fk;                        // concurrent z-layer launch and oblique-wire gather
    cudaGraphExec_t graph[6] = {};  // captured graphs of 2^k steps (k = 1..5) from parity 0
    int parity = 0;
    long step = 0;
    std::string err;
};

namespace {

int bfail(fdtd_batch *b, int code, const std::string &msg)
{
    if (b) b->err = msg;
    return code;
}

cudaError_t batch_launch(const fdtd_batch *b, int parity, int l, cudaStream_t s)
{
    fdtd::BatchArgs a{};
    a.doms = b->doms;
    a.item_start = b->item_start[l];
    a.n_domains = (int)b->grids.size();
    a.nitems = b->nitems[l];
    a.launch = l;
    a.parity = parity;
    a.work = b->work + 2 * l;
    a.err = b->errf;
    a.max_classes = b->max_classes;
    a.max_d = b->max_d;
    a.region = b->region[l];
    a.nh = b->nh[l];
    a.img = b->img;
    a.img_ref = b->img_ref;
    static const fdtd::SingleArgs none{};
    return fdtd::launch_step(none, a, b->grid[l], s);
}

cudaError_t batch_enqueue(fdtd_batch *b, int parity, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    const int nd = (int)b->grids.size();
    auto launch = [b, parity](int l) {
        return [b, parity, l](cudaStream_t st) {
            return l < b->n_launch && b->nitems[l] > 0 ? batch_launch(b, parity, l, st) : cudaSuccess;
        };
    };
    if (b->fk.side) {
        // side stream: the oblique wires' gather, then the z-layer launch
        auto side = [b, parity, nd, &launch](cudaStream_t st) {
            cudaError_t r = b->has_wires ? fdtd::launch_wire_gather_batch(b->edges, nd, parity, st) : cudaSuccess;
            if (r == cudaSuccess) r = launch(1)(st);
            return r;
        };
        e = b->fk.run(s, side, launch(0));
    } else {
        if (b->has_wires) e = fdtd::launch_wire_gather_batch(b->edges, nd, parity, s);
        for (int l = 0; l < b->n_launch && e == cudaSuccess; ++l) e = launch(l)(s);
    }
    if (e == cudaSuccess && b->has_edges) e = fdtd::launch_edges_batch(b->edges, nd, parity, b->has_wires, s);
    return e;
}

// n batch steps: graph replays of 32, 16, 8, 4 or 2 steps (each captured
// once, from parity 0) while the parity allows, direct launches otherwise
int batch_queue(fdtd_batch *b, int n)
{
    const int n0 = n;
    while (n > 0) {
        if (b->parity == 0 && n >= 2) {
            int k = 1;
            while (k < 5 && (2 << k) <= n) ++k;
            const int len = 1 << k;
            if (!b->graph[k]) {
                // all five sizes at once, so no later call pays a capture
                nvtxRangePushA("fdtd_batch_step graph capture");
                cudaError_t e = cudaSuccess;
                if (!b->cap) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
                for (int kk = 1; kk <= 5 && e == cudaSuccess; ++kk) {
                    cudaGraph_t graph = nullptr;
                    e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
                    if (e == cudaSuccess) {
                        for (int t = 0; t < (1 << kk) && e == cudaSuccess; ++t) e = batch_enqueue(b, t & 1, b->cap);
                        cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
                        if (e == cudaSuccess) e = e2;
                    }
                    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph[kk], graph, 0);
                    if (graph) cudaGraphDestroy(graph);
                    if (e != cudaSuccess) b->graph[kk] = nullptr;
                }
                nvtxRangePop();
                if (e != cudaSuccess) return bfail(b, FDTD_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
            }
            cudaError_t e = cudaGraphLaunch(b->graph[k], b->stream);
            if (e != cudaSuccess) return bfail(b, FDTD_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
            n -= len;
        } else {
            cudaError_t e = batch_enqueue(b, b->parity, b->stream);
            if (e != cudaSuccess) return bfail(b, FDTD_ECUDA, std::string("step launch: ") + cudaGetErrorString(e));
            b->parity ^= 1;
            n -= 1;
        }
    }
    b->step += n0;
    for (fdtd_grid *g : b->grids) {
        g->parity = b->parity;
        g->step = b->step;
    }
    return FDTD_OK;
}

}  // namespace

extern "C" {

int fdtd_batch_create(int n, fdtd_grid *const *grids, void *cuda_stream, fdtd_batch **out)
{
    if (!out || n < 1 || !grids) return FDTD_EINVAL;
    *out = nullptr;
    fdtd_batch *b = new (std::nothrow) fdtd_batch();
    if (!b) return FDTD_ENOMEM;
    b->stream = (cudaStream_t)cuda_stream;
    for (int q = 0; q < n; ++q) {
        fdtd_grid *g = grids[q];
        if (!g || !g->finalized) { delete b; return FDTD_ESTATE; }
        if (g->npoles) { delete b; return FDTD_EINVAL; }      // dispersive media run on their own
        if ((double)g->plane * g->nz >= 2147483647.0) { delete b; return FDTD_EINVAL; }  // 32-bit indices
        if (g->parity != grids[0]->parity || g->step != grids[0]->step) { delete b; return FDTD_ESTATE; }
        b->grids.push_back(g);
    }
    b->parity = grids[0]->parity;
    b->step = grids[0]->step;
    // launch sizing over all domains
    std::vector<int> starts[2];
    for (int l = 0; l < 2; ++l) starts[l].push_back(0);
    for (fdtd_grid *g : b->grids) {
        b->max_classes = std::max(b->max_classes, g->n_classes);
        b->max_d = std::max(b->max_d, g->d);
        b->n_launch = std::max(b->n_launch, g->n_launch);
        b->has_edges = b->has_edges || has_edge_work(g);
        b->has_wires = b->has_wires || !g->osegs.empty();
        for (int l = 0; l < 2; ++l) {
            const int items = l < g->n_launch ? g->lc[l].nitems : 0;
            starts[l].push_back(starts[l].back() + items);
            if (l < g->n_launch) b->region[l] = std::max(b->region[l], g->lc[l].region);
        }
    }
    int dev = 0, sms = 0, smem_per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    int max_smem = 0;
    for (int l = 0; l < b->n_launch && e == cudaSuccess; ++l) {
        b->nitems[l] = starts[l].back();
        b->nh[l] = 3;
        if (2 * (fdtd::step_smem_bytes(b->max_classes, b->max_d, b->region[l], 3) + 1024) > smem_per_sm &&
            2 * (fdtd::step_smem_bytes(b->max_classes, b->max_d, b->region[l], 2) + 1024) <= smem_per_sm)
            b->nh[l] = 2;
        max_smem = std::max(max_smem, fdtd::step_smem_bytes(b->max_classes, b->max_d, b->region[l], b->nh[l]));
    }
    for (int nh = 2; nh <= 3 && e == cudaSuccess; ++nh) e = ensure_smem(fdtd::step_kernel_ptr(nh, true, false), max_smem);
    for (int l = 0; l < b->n_launch && e == cudaSuccess; ++l) {
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &occ, fdtd::step_kernel_ptr(b->nh[l], true, false), fdtd::step_threads(),
            fdtd::step_smem_bytes(b->max_classes, b->max_d, b->region[l], b->nh[l]));
        if (e == cudaSuccess && occ < 1) { delete b; return FDTD_ECUDA; }
        b->grid[l] = std::max(1, std::min(sms * std::max(occ, 1), b->nitems[l]));
    }
    if (e != cudaSuccess) { delete b; return FDTD_ECUDA; }
    // device tables
    const size_t nd = b->grids.size();
    // staging images: per domain, launch and input parity its StepArgs, then
    // its class table rows spaced for max_classes, then its CPML profile rows,
    // exactly as the step kernel lays them out in shared memory
    std::vector<int4> img;
    std::vector<int2> img_ref(4 * nd);
    {
        const size_t tab_off = fdtd::step_tab_offset();
        for (size_t q = 0; q < nd && e == cudaSuccess; ++q) {
            fdtd_grid *g = b->grids[q];
            std::vector<float> table(g->n_classes * (size_t)fdtd::kNumCoef);
            e = cudaMemcpy(table.data(), g->table_d, table.size() * sizeof(float), cudaMemcpyDeviceToHost);
            const int d2 = 2 * g->d;
            const size_t bytes = tab_off + (size_t)b->max_classes * 48 + (g->d > 0 ? 3 * 2 * (size_t)d2 * 16 : 0);
            std::vector<char> im((bytes + 15) / 16 * 16, 0);
            float *tab = reinterpret_cast<float *>(im.data() + tab_off);
            for (int cl = 0; cl < g->n_classes; ++cl)
                for (int c = 0; c < 3; ++c) {
                    tab[cl * 12 + c] = table[cl * fdtd::kNumCoef + 6 + c];       // db
                    tab[cl * 12 + 4 + c] = table[cl * fdtd::kNumCoef + c];       // ca
                    tab[cl * 12 + 8 + c] = table[cl * fdtd::kNumCoef + 3 + c];   // cb
                }
            if (g->d > 0) {
                float *prof = tab + (size_t)b->max_classes * 12;
                const int n[3] = {g->nx, g->ny, g->nz};
                for (int u = 0; u < 3; ++u) {
                    const std::vector<float> pr = cpml_profile(g, n[u]);
                    for (int w = 0; w < fdtd::PR_COUNT; ++w)
                        for (int sl = 0; sl < d2; ++sl) {
                            const int i = sl < g->d ? sl : n[u] - d2 + sl;
                            prof[(((u * 2 + w / 3) * d2 + sl) << 2) + w % 3] = pr[(size_t)w * n[u] + i];
                        }
                }
            }
            for (int l = 0; l < 2; ++l)
                for (int par = 0; par < 2; ++par) {
                    std::memcpy(im.data(), &g->slot_h.a[l][par], sizeof(fdtd::StepArgs));
                    img_ref[(q * 2 + l) * 2 + par] = int2{(int)img.size(), (int)(im.size() / 16)};
                    const int4 *v = reinterpret_cast<const int4 *>(im.data());
                    img.insert(img.end(), v, v + im.size() / 16);
                }
        }
        if (e != cudaSuccess) { delete b; return FDTD_ECUDA; }
    }
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t at = off; off = align_up(off + bytes, 256); return at; };
    const size_t o_doms = take(nd * sizeof(fdtd::DomainSlot));
    const size_t o_s0 = take((nd + 1) * sizeof(int));
    const size_t o_s1 = take((nd + 1) * sizeof(int));
    const size_t o_edges = take(2 * nd * sizeof(fdtd::EdgeArgs));
    const size_t o_work = take(8 * sizeof(int));
    const size_t o_img = take(img.size() * sizeof(int4));
    const size_t o_ref = take(img_ref.size() * sizeof(int2));
    if (cudaMalloc(&b->mem, off) != cudaSuccess) { delete b; return FDTD_ENOMEM; }
    char *base = (char *)b->mem;
    b->doms = (fdtd::DomainSlot *)(base + o_doms);
    b->item_start[0] = (int *)(base + o_s0);
    b->item_start[1] = (int *)(base + o_s1);
    b->edges = (fdtd::EdgeArgs *)(base + o_edges);
    b->work = (int *)(base + o_work);
    b->errf = b->work + 4;
    b->img = (int4 *)(base + o_img);
    b->img_ref = (int2 *)(base + o_ref);
    std::vector<fdtd::DomainSlot> slots(nd);
    std::vector<fdtd::EdgeArgs> edges(2 * nd);
    for (size_t q = 0; q < nd; ++q) {
        slots[q] = b->grids[q]->slot_h;
        edges[2 * q] = b->grids[q]->edge_h[0];
        edges[2 * q + 1] = b->grids[q]->edge_h[1];
    }
    cudaStream_t s = b->stream;
    e = cudaMemsetAsync(b->mem, 0, off, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->doms, slots.data(), nd * sizeof(fdtd::DomainSlot), cudaMemcpyHostToDevice, s);
    for (int l = 0; l < 2 && e == cudaSuccess; ++l)
        e = cudaMemcpyAsync(b->item_start[l], starts[l].data(), (nd + 1) * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->edges, edges.data(), 2 * nd * sizeof(fdtd::EdgeArgs), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->img, img.data(), img.size() * sizeof(int4), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->img_ref, img_ref.data(), img_ref.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    // the grids' own work must be finished before the batch reads them
    for (fdtd_grid *g : b->grids)
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e == cudaSuccess && ((b->n_launch == 2 && b->nitems[0] > 0 && b->nitems[1] > 0) || b->has_wires))
        e = b->fk.init();
    if (e != cudaSuccess) { cudaFree(b->mem); delete b; return FDTD_ECUDA; }
    *out = b;
    return FDTD_OK;
}

int fdtd_batch_step(fdtd_batch *b, int n)
{
    if (!b) return FDTD_EINVAL;
    if (n < 0) return bfail(b, FDTD_EINVAL, "negative step count");
    nvtxRangePushA("fdtd_batch_step");
    const int rc = batch_queue(b, n);
    nvtxRangePop();
    return rc;
}

int fdtd_batch_synchronize(fdtd_batch *b)
{
    if (!b) return FDTD_EINVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, FDTD_ECUDA, std::string("synchronize: ") + cudaGetErrorString(e));
    int flag = 0;
    e = cudaMemcpy(&flag, b->errf, sizeof flag, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bfail(b, FDTD_ECUDA, "error flag read");
    if (flag) return bfail(b, FDTD_ETIMEOUT, "a bounded wait in the step kernel gave up");
    return FDTD_OK;
}

int fdtd_batch_launch_info(const fdtd_batch *b, int launch, int *ctas, int *items)
{
    if (!b || launch < 0 || launch > 1) return FDTD_EINVAL;
    if (ctas) *ctas = launch < b->n_launch ? b->grid[launch] : 0;
    if (items) *items = launch < b->n_launch ? b->nitems[launch] : 0;
    return FDTD_OK;
}

const char *fdtd_batch_last_error(const fdtd_batch *b) { return b ? b->err.c_str() : "null batch"; }

void fdtd_batch_destroy(fdtd_batch *b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    for (cudaGraphExec_t gr : b->graph)
        if (gr) cudaGraphExecDestroy(gr);
    if (b->cap) cudaStreamDestroy(b->cap);
    b->fk.destroy();
    if (b->mem) cudaFree(b->mem);
    delete b;
}

}  // extern "C"
