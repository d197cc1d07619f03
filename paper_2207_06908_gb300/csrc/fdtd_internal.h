// fdtd_internal.h -- structures shared by the host runtime and the kernels
// of the GB300 FDTD library (not part of the public C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace fdtd {

// Coefficients of one class, in this order (1/dx folded into cb and db):
//   ca_x ca_y ca_z  cb_x cb_y cb_z  db_x db_y db_z
constexpr int kNumCoef = 9;
constexpr int kMaxClasses = 256;

// Auxiliary CPML fields, one per (component, derivative axis), stored
// compactly: only the cells of their axis's two layers, indexed by the slab
// entry (0 .. d-1 the low layer, d .. 2d-1 the high one) along that axis --
// x [nz][ny][px] (px = 2d rounded up to a multiple of 4), y [nz][2d][pitch],
// z [2d][ny][pitch] -- so TMA boxes address them like the fields.
enum Psi {
    PSI_HY_X = 0, PSI_HZ_X, PSI_EY_X, PSI_EZ_X,
    PSI_HX_Y, PSI_HZ_Y, PSI_EX_Y, PSI_EZ_Y,
    PSI_HX_Z, PSI_HY_Z, PSI_EX_Z, PSI_EY_Z,
    PSI_COUNT
};

// 1D CPML profile per axis, n entries each, indexed by the cell index i:
//   E position (node i):      be, ce, kie
//   H position (node i + 1/2): bh, ch, kih
enum Prof { PR_BE = 0, PR_CE, PR_KIE, PR_BH, PR_CH, PR_KIH, PR_COUNT };

// Tile geometry of the step kernel, shared with the host (tensor-map boxes).
namespace geom {
constexpr int TX = 32, TY = 16;
constexpr int XO = 4;                        // box column of the tile's x0 (E, H)
constexpr int EBX = TX + 8, EBY = TY + 2;    // E box: x0-4 .. x0+TX+3, y0-1 .. y0+TY
constexpr int HBX = TX + 4, HBY = TY + 1;    // H box: x0-4 .. x0+TX-1, y0-1 .. y0+TY-1
constexpr int CXO = 16;                      // box column of x0 in the class box
constexpr int CBX = TX + 16, CBY = TY + 1;   // class box: x0-16 .. x0+TX-1
}  // namespace geom

// TMA descriptors of the current input buffers: E (E box), H (H box), class
// plus the CPML auxiliaries: z layer with the H box (HX_Z, HY_Z) and the
// tile box (EX_Z, EY_Z); x layer (HY_X, HZ_X | EY_X, EZ_X) with a box
// narrowed to the layer along x; y layer (HX_Y, HZ_Y | EX_Y, EZ_Y) with a
// box narrowed to the layer along y
struct TmaMaps {
    CUtensorMap e[3];
    CUtensorMap h[3];
    CUtensorMap c;
    CUtensorMap zh[2], ze[2];
    CUtensorMap xh[2], xe[2];
    CUtensorMap yh[2], ye[2];
};

// geometry of the staged CPML boxes (host-computed for the grid's layer)
struct PsiGeom {
    int w;                   // x-layer box width (slab entries, multiple of 4)
    int hy;                  // y-layer box height (slab rows)
    int xb, yb;              // bytes of one x / y box slot (128-aligned)
};

// Debye media: up to kMaxPoles poles per edge; per cell one record of
// [E component][pole]{cj, k, be} (E^{n+1} += cj J^n, J^{n+1} = k J^n +
// be (E^{n+1} - E^n)); record 0 = no dispersive component
constexpr int kMaxPoles = 4;
constexpr int kDebyeRec = 3 * kMaxPoles * 3;

struct SourceDesc {
    int comp;                // 0..2
    long long idx;           // element index in the field arrays
    float coef;              // -cb / dx of the edge
    int n_samples;
    long long sample_off;    // offset into the sample table
    long long jidx;          // element index in the Debye current arrays, or -1
    float be[kMaxPoles];     // be of the edge's poles (dispersive edge)
    int hard;                // ideal voltage source: samples are volts, E is set to vcoef * V
    float vcoef;             // -1 / dx
};

struct StepArgs {
    int nx, ny, nz;
    int pitch;               // row pitch in elements (multiple of 4)
    long long plane;         // plane pitch in elements (pitch * ny)
    const float *Ein[3];
    const float *Hin[3];
    float *Eout[3];
    float *Hout[3];
    const uint8_t *cls;      // class per cell, same pitch as the fields
    const float *table;      // [n_classes][kNumCoef]
    int n_classes;
    int d;                   // CPML cells (0 = none)
    const float *prof[3];    // per axis: PR_COUNT arrays of n_axis floats
    const float *psi_in[PSI_COUNT];  // compact: x [nz][ny][px], y [nz][2d][pitch], z [2d][ny][pitch]
    float *psi_out[PSI_COUNT];
    int px;                  // row pitch of the x-layer auxiliaries (2d rounded up to a multiple of 4)
    int kz;                  // planes per z block of a work item
    int zlo, zhi;            // planes of this launch: [zlo, zhi) and [zlo2, zhi2)
    int zlo2, zhi2;
    int ncx, ncy;            // column tiles along x, y
    int nitems;              // (z blocks) x (column tiles)
    PsiGeom pg;
    int region;              // bytes of the staged-auxiliary region this domain needs
    int ox, oy;              // byte offsets of the x and y box groups in that region
    int zxy;                 // 1: stage the z layer together with x / y
    const int *col_order;    // [ncx * ncy] column tile of each position in a z block (costliest first)
    // current sources applied in the E update of the items that own their
    // edges (single-grid steps only; n_isrc = 0: the source/probe kernel
    // applies them): source q lies in launch isrc_loc[q].x, item .y
    int n_isrc;
    const int2 *isrc_loc;
    const SourceDesc *src;
    const float *samples;
    const long long *step;   // device step counter; this step's sample is *step + step_t
    int step_t;
    int *bounds;             // bounds-checked build: {first site, count} of skipped accesses
};

// One domain of a step launch, in device memory (the launch reads the
// arguments and TMA descriptors of the domain each work item belongs to).
struct DomainSlot {
    TmaMaps m[2];            // descriptors of input parity 0, 1
    StepArgs a[2][2];        // [launch: 0 = planes between the z layers, 1 = z layers][input parity]
};

// One domain passed in the kernel's own parameters (single-grid launches).
struct SingleArgs {
    TmaMaps m;
    StepArgs a;
};

// One launch of the step kernel over one or more domains (doms == nullptr:
// the single domain of SingleArgs, items 0 .. nitems-1).  Work items of
// domain d are the global items item_start[d] .. item_start[d+1]-1.
struct BatchArgs {
    const DomainSlot *doms;
    const int *item_start;   // [n_domains + 1]
    int n_domains;
    int nitems;
    int launch;              // 0 or 1 (selects StepArgs a[launch])
    int parity;              // input parity of this step
    int *work;               // [2] work counter, finished-CTA counter (self-resetting)
    int *err;                // set to 1 when a bounded wait gave up
    int max_classes, max_d;  // shared-memory sizing over the domains
    int region;              // staged-auxiliary region (max over the domains)
    int nh;                  // slots of the H / class / CPML ring (2 or 3)
    int wide;                // single grid of 2^31 elements or more: 64-bit field indices
    // batches: per (domain, launch, parity) {offset, length} in int4 of the
    // domain's staging image in img -- its StepArgs, table rows and CPML
    // profile rows in the layout of their shared-memory copy
    const int4 *img;
    const int2 *img_ref;
};

// shared-memory layout of a domain's staging image (and of the step
// kernel's copy): StepArgs, then from byte step_tab_offset() the class table
// (max_classes rows of 12 floats: {db xyz, 0}, {ca xyz, 0}, {cb xyz, 0}),
// then the CPML profiles ([axis][E, H][2d] x {b, c, 1/kappa, 0})



struct DebyeArgs {
    const float *Ein[3];     // E^n (the step's input buffers)
    float *Eout[3];          // E^{n+1} from the step kernels, completed in place
    float *J;                // [3 * npoles][jstride] polarisation currents, box layout
    long long jstride;       // elements per current array (box planes x plane)
    int npoles;
    const uint8_t *dcls;     // per box element: record index
    const float *table;      // [n_rec][kDebyeRec]
    int n_rec;
    long long off;           // field element index of the box's first element
};

struct ProbeDesc {
    int kind, axis;
    int i, j, k, n_edges;
};

// Oblique thin wires (Sec. 2.3, the Guiffaut formalism in Holland-Simpson
// form): segment currents I_s (t_{n+1/2}) and node charges Q_m (t_n).
struct OSeg {
    int a, b;                // end nodes; I flows a -> b
    int e0, ne;              // gather edges e0 .. e0+ne-1
    int s0, ns;              // its delta-gap sources s0 .. s0+ns-1
    float cI, cIV;           // dt / L', dt / (L' dl)
    float rk, rd;            // series resistance R of its sources, k = cIV R / 2:
                             // I^{n+1/2} = rk I^{n-1/2} + rd (increment), rk = (1-k)/(1+k), rd = 1/(1+k)
};
struct OEdge {
    long long idx;           // element index in the field arrays
    int comp;                // E component
    float wg;                // E_s += wg E
};
struct OScat {               // one coupled edge: E -= sum over its terms of ws I_seg
    long long idx;
    int comp;
    int t0, nt;              // terms t0 .. t0+nt-1, in segment order
};
struct OTerm {
    int seg;
    float ws;
};
struct ONode {
    // in-cell medium: K Q = e0 V + sum_p P_p; Q^{n+1} = Q^n + dt (net current
    // in) - (cs / K)(V^{n+1} + V^n); P_p^{n+1} = pa_p P_p^n + pb_p (V^{n+1} + V^n)
    float K, e0, cs;
    float pa[4], pb[4];      // Debye poles of the node's medium (0: none)
    int grounded;
    int adj0, nadj;          // adjacency entries (segment << 1 | current flows in)
};
struct OSrc {
    int n;                   // samples (V at t_n)
    long long off;           // offset into the wire sample table
    float cIV;               // dt / (L' dl) of its segment
};
constexpr int kWireChunk = 4096;      // gather entries the source/probe kernel stages at a time
struct WireArgs {
    const OSeg *seg;
    int n_seg;
    const int *chunk;        // [n_chunk + 1] first segment of each chunk of whole segments whose
    int n_chunk;             // gather entries fit kWireChunk, then n_seg
    const OEdge *edge;
    const OScat *scat;
    int n_scat;
    const OTerm *term;
    const ONode *node;
    int n_node;
    const int *adj;
    float *I, *Q, *V;        // segment currents, node charges and in-cell potentials
    float *P;                // [n_node][4] node polarisations (Debye media)
    const OSrc *src;
    const float *samples;
};

struct EdgeArgs {
    int nx, ny, nz, pitch;
    long long plane;
    float dx, dt;
    float *E[3];             // fields after the stencil (t_{n+1}, t_{n+1/2})
    const float *H[3];
    const SourceDesc *src;
    int n_src;
    const float *samples;
    const ProbeDesc *probes;
    int n_probes;
    float *probe_out;        // [n_probes][capacity]
    int capacity;
    long long *step;         // device step counter
    float *J;                // Debye currents (sources on dispersive edges), or null
    long long jstride;
    int npoles;
    const float *Ein[3];     // E^n, the step's input (oblique wires read it)
    WireArgs w;              // oblique wires (n_seg = 0: none)
    int wire_done;           // the wires' scatter and charges ran before the Debye kernel
    int step_t;              // this launch serves step *step + step_t
    int advance;             // 1: set *step to that step + 1 when done
    int skip_src;            // the current sources ran in the step kernel
    int *bounds;             // bounds-checked build: {first site, count} of skipped accesses
};

// Bounds-checked build (compiled with -DFDTD_BOUNDS, a debugging aid): the
// global accesses of the step and source/probe kernels test their element
// index against the array's extent; an access outside it is skipped and
// counted in bounds[1], the first site recorded in bounds[0].  In the
// release build the test is the constant true.
#ifdef FDTD_BOUNDS
__device__ __forceinline__ bool in_bounds(long long idx, long long n, int site, int *bounds)
{
    if (idx >= 0 && idx < n) return true;
    if (bounds) {
        atomicCAS(bounds, 0, site);
        atomicAdd(bounds + 1, 1);
    }
    return false;
}
#else
__device__ __forceinline__ bool in_bounds(long long, long long, int, int *) { return true; }
#endif

// the six field arrays of one state (Ex Ey Ez Hx Hy Hz)
struct FieldPtrs {
    const float *p[6];
};

// fdtd_watch.cu: sets *flag to 1 if any of the six arrays (n_elems floats
// each, a multiple of 4, 16-byte aligned) holds a NaN or an infinity
cudaError_t launch_finite_check(const FieldPtrs &f, long long n_elems, int *flag, int blocks, cudaStream_t s);

// fdtd_step.cu
cudaError_t launch_step(const SingleArgs &one, const BatchArgs &b, int grid, cudaStream_t s);
int step_tile_x();
int step_tile_y();
int step_threads();
int step_smem_bytes(int n_classes, int d, int region, int nh);
int step_tab_offset();      // bytes from the start of the StepArgs copy to the class table
PsiGeom step_psi_geom(int d, int nx, int ny);
// region size and box-group offsets for a launch that stages z alone
// (zxy = 0) or z together with the x / y layers (zxy = 1)
void step_region(const PsiGeom &pg, int zxy, int *region, int *ox, int *oy);
const void *step_kernel_ptr(int nh, bool batch, bool wide);
// fdtd_edges.cu
cudaError_t launch_edges(const EdgeArgs &a, cudaStream_t s);
// oblique wires: segment currents to t_{n+1/2}; needs only the step's inputs,
// so it may run concurrently with the step kernels, and before launch_edges
cudaError_t launch_wire_gather(const EdgeArgs &a, cudaStream_t s);
// oblique wires in Debye media: their scatter into E^{n+1} and node charges,
// before the dispersive-media kernel (which then sees the wire currents)
cudaError_t launch_wire_finish(const EdgeArgs &a, cudaStream_t s);
cudaError_t launch_debye(const DebyeArgs &a, cudaStream_t s);
// one CTA per domain: e[2 * d + parity]; wires: some domain has oblique wires
cudaError_t launch_edges_batch(const EdgeArgs *e, int n_domains, int parity, bool wires, cudaStream_t s);
// one CTA per domain, the oblique wires' segment currents (domains without
// wires return at once); may run concurrently with the step kernels
cudaError_t launch_wire_gather_batch(const EdgeArgs *e, int n_domains, int parity, cudaStream_t s);

}  // namespace fdtd

struct fdtd_grid;
namespace fdtd {
// fdtd_runtime.cu, for fdtd_noalloc.cu
int step_with_scratch(fdtd_grid *g, int n, int *scratch, int scratch_ints);
int set_error(fdtd_grid *g, int code, const char *msg);
}  // namespace fdtd
