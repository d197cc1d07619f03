/*
 * fdtd.h -- C ABI of the GB300 (sm_103a) FDTD library.
 *
 * The library advances Maxwell's curl equations (Kuklin, "elecode",
 * arXiv 2207.06908, Sec. 2.1, Eq. maxwell / maxwelle / maxwellh) on a
 * uniform cubic Yee grid with the staggered updates of Eq. fdtdex and
 * Eq. fdtdhx, in FP32 on one GPU.  Per-cell eps, sigma, mu come from a
 * uint8 material map; thin wires (Sec. 2.3), ideal current sources
 * (Sec. 2.1, "sources"), a CPML absorbing layer (Sec. 2.2) and the voltage /
 * current probes of the Sec. 4 model files ("calculate") are supported.
 *
 * Conventions for every call:
 *   - Return value: FDTD_OK (0) or a negative FDTD_E* code.  Nothing throws
 *     across the ABI.  fdtd_last_error() gives a one-line reason.
 *   - Host arrays passed in are copied before the call returns; the caller
 *     keeps ownership.  Host arrays passed out are written by the call.
 *   - A grid handle is owned by the library and freed by fdtd_destroy().
 *   - Mutators (set_materials, add_*) fail with FDTD_ESTATE after
 *     fdtd_finalize(); step/read/get/set fail with FDTD_ESTATE before it.
 *   - Indices are node indices: node (i,j,k) sits at (i dx, j dx, k dx),
 *     0 <= i <= nx.  Cell (i,j,k) is the cube above node (i,j,k) and owns
 *     the six components Ex(i+1/2,j,k) Ey(i,j+1/2,k) Ez(i,j,k+1/2)
 *     Hx(i,j+1/2,k+1/2) Hy(i+1/2,j,k+1/2) Hz(i+1/2,j+1/2,k).
 *   - Field arrays exchanged with the host are nx*ny*nz floats, x fastest
 *     (index (k*ny + j)*nx + i), entry = the component owned by that cell.
 *     E is at t_n, H at t_{n-1/2} when n steps have been taken.
 *   - The outer boundary is PEC: tangential E on the six faces is zero.
 *     With a CPML the layer sits inside the grid, next to that wall.
 *   - Work is queued on the CUDA stream given at creation; calls that return
 *     host data synchronise that stream first.
 */
#ifndef FDTD_GB300_FDTD_H
#define FDTD_GB300_FDTD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fdtd_grid fdtd_grid;

/* One material: relative permittivity, conductivity (S/m), relative
 * permeability.  eps_r > 0, sigma >= 0, mu_r > 0. */
typedef struct {
    double eps_r;
    double sigma;
    double mu_r;
} fdtd_material;

/* CPML layer (Sec. 2.2, convolutional PML of Roden and Gedney, CFS form).
 * cells: thickness in cells on each of the six faces (0 = plain PEC box);
 * order: polynomial grading m of sigma and kappa; kappa_max >= 1;
 * alpha_max >= 0 (S/m) with grading order alpha_order;
 * sigma_max <= 0 selects 0.8 (m + 1) / (eta0 dx). */
typedef struct {
    int cells;
    double order;
    double kappa_max;
    double alpha_max;
    double alpha_order;
    double sigma_max;
} fdtd_cpml;

enum {
    FDTD_OK = 0,
    FDTD_EINVAL = -1,     /* bad argument, index out of range */
    FDTD_ECOURANT = -2,   /* Courant number outside (0, 1] */
    FDTD_ENOMEM = -3,     /* host or device allocation failed, or arena too small */
    FDTD_ECUDA = -4,      /* a CUDA call failed */
    FDTD_ECLASSES = -5,   /* more than 256 distinct coefficient classes */
    FDTD_ETIMEOUT = -6,   /* a bounded device wait ran out */
    FDTD_EDIVERGED = -7,  /* the watchdog found a NaN or an infinity in the fields */
    FDTD_ESTATE = -8      /* call not allowed in the grid's current state */
};

enum {
    FDTD_PROBE_V = 0,     /* voltage -sum E_axis dx over n_edges edges from node (i,j,k) along +axis, at t_{n+1} */
    FDTD_PROBE_I = 1,     /* current: loop integral of H around the edge from node (i,j,k) along +axis, at t_{n+1/2} */
    FDTD_PROBE_E = 2,     /* E component `axis` owned by cell (i,j,k), at t_{n+1} */
    FDTD_PROBE_H = 3,     /* H component `axis` owned by cell (i,j,k), at t_{n+1/2} */
    FDTD_PROBE_WIRE = 4,  /* current of one oblique-wire segment, at t_{n+1/2} (fdtd_add_wire_probe) */
    FDTD_PROBE_WIRE_V = 5 /* in-cell potential of an oblique-wire node, at t_{n+1} (fdtd_add_wire_node_probe) */
};

/* Create a grid of nx*ny*nz cells of edge dx metres.  The time step is
 * dt = courant * dx / (c0 sqrt 3), the Courant limit of the cubic Yee grid
 * (Sec. 2.1) scaled by courant in (0, 1].  cpml may be NULL (PEC box).
 * cuda_stream: a cudaStream_t (NULL = the legacy default stream) on which
 * all device work of this grid is queued.  Every material starts as vacuum.
 * nx, ny, nz >= 2 (>= 2*cells + 2 with a CPML).  With a CPML each of its
 * compact auxiliary arrays (the layer cells of one axis) must stay below
 * 2^31 elements (FDTD_EINVAL otherwise; about 10^4 cells per side for a
 * 10-cell layer).  *out receives the handle. */
int fdtd_create_grid(int nx, int ny, int nz, double dx, double courant,
                     const fdtd_cpml *cpml, void *cuda_stream, fdtd_grid **out);

/* Material map (Sec. 4 model files, "block"): cell_material is nx*ny*nz
 * bytes, x fastest, each < n_materials; table holds n_materials (1..256)
 * entries.  E edges take the mean eps, sigma of the four cells around them,
 * H faces the mean mu of the two cells on either side. */
int fdtd_set_materials(fdtd_grid *g, const uint8_t *cell_material,
                       const fdtd_material *table, int n_materials);

/* Debye poles of material `material` (the paper's "Dispersive media"
 * subsection: a multi-term Debye permittivity eps(w) = eps_inf + sum_p
 * deps_p / (1 + j w tau_p), eps_inf and the static sigma being the
 * material's eps_r and sigma, simulated by the auxiliary differential
 * equation method the paper cites).  delta_eps[p] (relative, >= 0) and
 * tau[p] (s, > 0) for p < n_poles <= 4; a later call replaces the poles.
 * Before fdtd_finalize (FDTD_ESTATE after), FDTD_EINVAL for bad values.
 * Each E edge takes, per pole index, the mean of its four cells' deps (zero
 * for a cell without the pole) and their deps-weighted mean tau; a thin
 * wire scales eps, sigma and every deps of its radial edges by its factor.
 * Grids with poles cannot join a batch (fdtd_batch_create: FDTD_EINVAL). */
int fdtd_set_debye(fdtd_grid *g, int material, int n_poles, const double *delta_eps, const double *tau);

/* Thin wire (Sec. 2.3; "wire(thin, ...)" in the Sec. 4 model files) along
 * one axis from node (i0,j0,k0) to node (i1,j1,k1), i1>i0 or j1>j0 or k1>k0
 * with the other two coordinates equal and strictly inside the grid
 * (1..n-1).  The on-wire E edges become PEC.  Radius 0 < radius <= 0.23 dx:
 * the radial E at each wire node take eps, sigma times
 * m = ln(dx / 0.23 dx) / ln(dx / radius) and every H those E read takes
 * mu / m.  Where two wires share a component the smaller m is used.
 * *wire_id (may be NULL) receives the wire's index. */
int fdtd_add_wire(fdtd_grid *g, int i0, int j0, int k0, int i1, int j1, int k1,
                  double radius, int *wire_id);

/* Thin wire between two arbitrary nodes (i0,j0,k0) and (i1,j1,k1) as a
 * staircase of grid-aligned wires (the staircase wire model the paper lists
 * among its thin-wire techniques, Sec. 2.3): from the first node each unit
 * step goes along the axis least advanced towards the second node,
 * |c_u - a_u| / |b_u - a_u| smallest, ties to the lowest axis; each run of
 * steps along one axis is one fdtd_add_wire() wire of the given radius.
 * Wires that meet at a node form a junction (the thinner wire's factor
 * applies where they share a component).  On an error (as fdtd_add_wire)
 * no wire of the path is kept.  *n_segments (may be NULL) receives the
 * number of wires added. */
int fdtd_add_wire_path(fdtd_grid *g, int i0, int j0, int k0, int i1, int j1, int k1, double radius,
                       int *n_segments);

/* Oblique thin wire (Sec. 2.3: the Guiffaut formalism the paper cites for
 * arbitrarily oriented wires and multiwire junctions; the paper prints none
 * of its equations, and this is the Holland-Simpson form of it).  A straight
 * wire from point (x0,y0,z0) to (x1,y1,z1) in node units (node (i,j,k) sits
 * at (i dx, j dx, k dx); any real coordinates in [0, n] per axis), length
 * >= 0.5 cell, radius 0 < radius <= 0.1 dx metres, split into
 * max(1, round(length in cells)) equal segments.  It carries its own
 * unknowns: a current per segment (t_{n+1/2}) and a charge per node (t_n),
 * with in-cell inductance, capacitance and leakage per unit length
 * mu ln(R/a) / (2 pi), 2 pi eps / ln(R/a), 2 pi sigma / ln(R/a), R the
 * radius at which the grid itself sees a line current at the segment's
 * sub-cell position (from the square-lattice Green's function), and the
 * medium of the cell holding the segment's centre or the node.  The grid
 * and the wire exchange E^n and the segment currents through the same edge
 * shares, those of the charge-conserving (Villasenor-Buneman) deposition of
 * the straight path between the segment's end nodes.  An end point equal
 * (within 1e-9) to a node of an earlier oblique wire joins that node
 * (junction: the currents of all segments at a node change its charge).  A
 * node on an outer wall is grounded (potential 0), and so is a node on the
 * node line of an axis-aligned wire (fdtd_add_wire, added before or after):
 * it joins that conductor, its charge handed to the grid, where the PEC
 * line carries it.  In Debye media the
 * in-cell capacitance takes the node medium's poles: K Q = eps0 eps_inf V +
 * sum_p P_p, K = ln(R/a) / (2 pi dl), tau_p dP_p/dt + P_p = eps0 deps_p V,
 * with the conduction sigma V K drawn from the charge.  Inside a CPML a wire
 * is a matched lossy line (series resistance and shunt conductance per unit
 * length L' nu and C' nu, nu = sum_u t_u^2 sigma_u / (kappa_u eps0) at the
 * segment, t its direction), so a wire may run into the layer and end
 * there.  Thick wires lower the
 * stable Courant number (fdtd_wire_courant_limit).  In a batch each domain's
 * wires run as when it steps alone.  *wire_id (may be NULL) receives the
 * index. */
int fdtd_add_oblique_wire(fdtd_grid *g, double x0, double y0, double z0, double x1, double y1, double z1,
                          double radius, int *wire_id);

/* Delta-gap EMF in segment `segment` (0-based from the wire's first point)
 * of oblique wire `wire_id`, in series with r_internal >= 0 ohm (a lightning
 * channel: the channel impedance): voltage[n] volts at t_n (0 after the last
 * sample) drive the segment's current from its first towards its second
 * point, L' dl dI/dt = E_s dl - (V_b - V_a) + V - r I with the r I term at
 * the mean of the two half steps.  voltage (n doubles, host) is copied and
 * rounded to FP32.  *source_id (may be NULL) receives the index among such
 * sources. */
int fdtd_add_wire_voltage_source(fdtd_grid *g, int wire_id, int segment, double r_internal, const double *voltage,
                                 int n, int *source_id);

/* Probe of the current of one oblique-wire segment at t_{n+1/2} (positive
 * from the wire's first point towards its second), read with
 * fdtd_read_probes; probe ids are shared with fdtd_add_probe. */
int fdtd_add_wire_probe(fdtd_grid *g, int wire_id, int segment, int *probe_id);

/* Probe of the in-cell potential Q / (C' dl) of the oblique-wire node at
 * point (x, y, z) (node units; it must be a node of a wire added earlier),
 * at t_{n+1}.  The grid does not hold that part of a thin wire's potential:
 * a voltage from the grid to the wire is a FDTD_PROBE_V path ending at the
 * node plus this probe. */
int fdtd_add_wire_node_probe(fdtd_grid *g, double x, double y, double z, int *probe_id);

/* Largest Courant number at which the grid's oblique wires keep the
 * coupled leapfrog stable: min over segments of
 * 1 / sqrt(1 + 2 |w|^2 exp(-1.89 ln(R/a))), |w|^2 the sum of the squared
 * edge shares of the segment (1 for a segment along a node line), a bound
 * set below the measured stability limit of wires along node lines.  1 when
 * there are none.  fdtd_finalize fails with FDTD_ECOURANT when the grid's
 * courant exceeds it.  Host only; any time before or after finalize. */
int fdtd_wire_courant_limit(const fdtd_grid *g, double *courant);

/* Number of oblique-wire segments and nodes (all wires, in the order
 * added; a wire's segments are consecutive, its interior nodes follow its
 * first point's node unless that point joined an earlier node). */
int fdtd_wire_counts(const fdtd_grid *g, int *n_segments, int *n_nodes);

/* Oblique-wire state after fdtd_finalize: I = segment currents of the last
 * half step (A, n_segments floats), Q = node charges (C, n_nodes floats);
 * host buffers.  get synchronises the grid's stream; set writes grounded
 * nodes as 0 and starts every node without medium polarisation. */
int fdtd_get_wire_state(fdtd_grid *g, float *I, float *Q);
int fdtd_set_wire_state(fdtd_grid *g, const float *I, const float *Q);

/* Current source (Sec. 2.1 sources: ideal and non-ideal current sources;
 * "source(current, ...)" in the Sec. 4 model files) on the edge from node
 * (i,j,k) along +axis (0,1,2): J = I / dx^2 along +axis, I(t_{n+1/2}) =
 * current[n] for n < n_samples and 0 after.  The transverse node
 * coordinates must lie in 1..n-1.  r_internal (ohm): 0 = ideal; > 0 = the
 * source's internal resistance in parallel, an extra conductivity
 * 1 / (r_internal dx) on the edge.  Samples are rounded to FP32.
 * *source_id (may be NULL) receives the index; voltage sources share the
 * numbering. */
int fdtd_add_source(fdtd_grid *g, int i, int j, int k, int axis, double r_internal,
                    const double *current, int n_samples, int *source_id);

/* Voltage source across the edge from node (i,j,k) along +axis (Sec. 2.1:
 * ideal and non-ideal voltage sources), its voltage V = -E dx (the sign of
 * a voltage probe on that edge).  r_internal = 0: ideal, E^{n+1} of the edge
 * is set to -voltage[n] / dx after the step (voltage[n] = V(t_{n+1}));
 * r_internal > 0: in series with that resistance, applied as its Norton
 * equivalent, a current voltage[n] / r_internal (at t_{n+1/2}) in parallel
 * with r_internal.  Two ideal sources on one edge: the later one applies.
 * Errors as fdtd_add_source. */
int fdtd_add_voltage_source(fdtd_grid *g, int i, int j, int k, int axis, double r_internal, const double *voltage,
                            int n_samples, int *source_id);

/* Lumped resistor and / or capacitor on the edge from node (i,j,k) along
 * +axis (the paper's lumped circuit elements, in the form of the textbook it
 * cites): edge current E dx / R and C dx dE/dt, i.e. an extra conductivity
 * 1 / (R dx) and permittivity C / dx on that edge (added after any thin-wire
 * factor).  resistance (ohm) and capacitance (F) >= 0, 0 = absent, not both
 * 0; several elements on one edge add in parallel.  FDTD_EINVAL for bad
 * values or an edge on a wall; FDTD_ESTATE after fdtd_finalize. */
int fdtd_add_lumped(fdtd_grid *g, int i, int j, int k, int axis, double resistance, double capacitance,
                    int *element_id);

/* Probe (Sec. 4 model files, "calculate(voltage|current, ...)"), one of
 * FDTD_PROBE_*.  For FDTD_PROBE_V, n_edges >= 1 edges from node (i,j,k)
 * along +axis; ignored otherwise.  FDTD_PROBE_I needs the two transverse
 * node coordinates >= 1.  *probe_id (may be NULL) receives the index. */
int fdtd_add_probe(fdtd_grid *g, int kind, int i, int j, int k, int axis, int n_edges,
                   int *probe_id);

/* Planes per work item of the step kernel (the depth of a 32x16 column
 * tile; 0 = the default 16).  Tuning only; results do not depend on it.
 * Before fdtd_finalize(); FDTD_EINVAL outside 0..256. */
int fdtd_set_block(fdtd_grid *g, int planes);

/* fdtd_set_watchdog: the divergence watchdog of fdtd_step().  The leapfrog
 * of Sec. 2.1 is stable only under the Courant bound; an unstable run grows
 * without bound, overflows FP32 and spreads NaN.  Every time the grid's
 * step count crosses a multiple of `every` during fdtd_step() (checked after
 * each graph replay or direct step), one streaming kernel reads the
 * six field arrays on the grid's stream and sets a device flag if any value
 * is a NaN or an infinity; the next fdtd_synchronize() (and every call that
 * synchronises: fdtd_read_probes, fdtd_get_field, ...) returns
 * FDTD_EDIVERGED and clears the flag, so a grid that keeps diverging
 * reports again at the next check.  A check reads 48 bytes per cell once;
 * with the default period of 1024 steps that is under 0.1 % of the steps'
 * traffic.  every = 0 turns the watchdog off.  Batches and
 * fdtd_step_noalloc() run no check.  Any time; FDTD_EINVAL if every < 0. */
int fdtd_set_watchdog(fdtd_grid *g, int every);

/* fdtd_bounds_report: the record of the bounds-checked build (a debugging
 * aid with no counterpart in the paper: the library compiled with
 * -DFDTD_BOUNDS, e.g. by _build.build_bounds()).  In that build every
 * global access of the step and source/probe kernels (field, CPML auxiliary,
 * source, probe and oblique-wire edge indices) tests its element index
 * against the array's extent and skips an access outside it.  The
 * grid's record holds the number of skipped accesses (*count) and the site
 * of the first (*site: 1 H store, 2 E store, 3 CPML auxiliary store, 4 CPML
 * auxiliary read, 5 in-kernel source, 6 source edge, 7 probe read, 8 wire
 * gather, 9 wire scatter).  Synchronises.  Returns FDTD_OK in the
 * bounds-checked build, 1 in the release build (nothing is checked there and
 * the record stays zero). */
int fdtd_bounds_report(fdtd_grid *g, int *site, int *count);

/* Device bytes fdtd_finalize() needs for probe_capacity recorded steps. */
int fdtd_arena_bytes(const fdtd_grid *g, int probe_capacity, size_t *bytes);

/* Build the coefficient classes, upload everything and zero the fields.
 * probe_capacity: number of steps recorded per probe (steps beyond it are
 * not recorded).  arena: device memory of at least fdtd_arena_bytes()
 * bytes, 256-byte aligned, owned by the caller and kept alive until
 * fdtd_destroy(); NULL makes the library allocate (and free) its own.
 * Fails with FDTD_ECLASSES if more than 256 distinct coefficient sets
 * occur. */
int fdtd_finalize(fdtd_grid *g, int probe_capacity, void *arena, size_t arena_bytes);

/* Queue n full time steps (H to n+1/2, E to n+1 with the sources, probes)
 * on the grid's stream: replays of captured CUDA graphs of 32, 16, 8, 4 and
 * 2 steps (each captured on first use), a lone step launched directly.
 * Returns launch errors only; does not synchronise. */
int fdtd_step(fdtd_grid *g, int n);

/* Wait for the grid's queued work; reports asynchronous CUDA errors. */
int fdtd_synchronize(fdtd_grid *g);

/* Size, in ints, of the device array fdtd_step_noalloc() uses as scratch. */
#define FDTD_NOALLOC_SCRATCH_INTS 64

/* fdtd_step_noalloc: the same n time steps as fdtd_step(), for callers that
 * cannot allocate device memory.  The paper has no counterpart: this is a
 * library entry point, not part of the method.
 *
 * Who needs it: a caller whose device memory is owned entirely by another
 * allocator (a framework's caching pool that must not be bypassed), a
 * real-time loop that cannot afford cudaMalloc's latency and implicit
 * synchronisation, or a process held to a fixed device-memory budget.  Such
 * a caller hands fdtd_finalize() an arena it obtained elsewhere and steps
 * with this function, which calls no cudaMalloc, cudaFree or other
 * allocating routine and never builds a CUDA graph: it queues plain kernel
 * launches (and one cudaMemsetAsync) on the grid's stream.
 *
 * The step kernel's scratch -- two work-distribution counters per launch and
 * the flag of a bounded wait that gave up, at most 5 ints today -- lives in
 * a file-scope device array of FDTD_NOALLOC_SCRATCH_INTS ints (256 bytes)
 * that every GPU which loads the library holds until the process exits.
 * The first call on a device looks the array's device address up
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call on a device shares the array and
 * keeps the last call's contents: the counters sit at the start of the
 * array and each call clears them on the grid's stream before its first
 * launch; the error flag is the array's last int, the same slot for every
 * grid, which no call clears on entry.  fdtd_synchronize() on a grid that
 * used this entry point reads the flag and clears it on the grid's stream.
 * Because the flag is shared, that call reports a timeout of any earlier
 * fdtd_step_noalloc() call on the device that no fdtd_synchronize() has
 * reported yet, whichever grid it stepped: synchronise each grid after its
 * own calls to tell whose steps gave up.  Calls that overlap on the GPU
 * (grids stepped through this entry point on different streams at the same
 * time) race on the counters.
 *
 * Returns FDTD_EINVAL if the grid needs more scratch than the array holds,
 * FDTD_ESTATE before fdtd_finalize(), FDTD_ECUDA on a launch error. */
int fdtd_step_noalloc(fdtd_grid *g, int n);

/* Copy count recorded samples of one probe, starting at step first_step,
 * to host_out (count floats).  Synchronises. */
int fdtd_read_probes(fdtd_grid *g, int probe_id, int first_step, int count, float *host_out);

/* Copy one component (0..5 = Ex Ey Ez Hx Hy Hz) to / from a host array of
 * nx*ny*nz floats.  Synchronises. */
int fdtd_get_field(fdtd_grid *g, int component, float *host_out);
int fdtd_set_field(fdtd_grid *g, int component, const float *host_in);

/* Device address, row pitch (elements) and plane pitch (elements) of the
 * current buffer of one component, for device-side consumers.  The address
 * changes after every step (the update ping-pongs between two buffers). */
int fdtd_field_device(fdtd_grid *g, int component, void **dptr, int *row_pitch,
                      size_t *plane_pitch);

/* ---- batched engine -------------------------------------------------
 * Many independent finalized grids (domains of different sizes, media,
 * wires, layers) advanced together -- the soil and grounding sweeps of
 * Sec. 4.1.  Every step is one persistent launch of the step kernel over the
 * work items of all domains (plus one over their CPML z-layer planes when
 * they have a CPML) and one source / probe launch with a CTA per domain
 * (which also adds the oblique wires' currents to E and updates their node
 * charges); when a domain has oblique wires, a launch with a CTA per domain
 * takes their segment currents to t_{n+1/2} beside the step kernel.
 * fdtd_batch_step replays captured CUDA graphs of 32, 16, 8, 4 and 2
 * steps (each captured on first use) and launches a lone step directly.
 * The results are those of stepping each grid alone with fdtd_step. */
typedef struct fdtd_batch fdtd_batch;

/* grids: n_grids finalized grids, all at the same step count, on the current
 * device; the batch reads their device state and keeps pointers to them (they
 * must outlive it and must not be stepped by other calls meanwhile).
 * cuda_stream: the stream the batch queues on.  Allocates a small device
 * table (about 16 KB per domain: launch arguments, tensor maps and the
 * staging images the step kernel copies into shared memory).  FDTD_ESTATE
 * if a grid is not finalized or the step counts differ; FDTD_EINVAL for a
 * grid with Debye poles or a grid of 2^31 cells or more (batch domains use
 * 32-bit indices). */
int fdtd_batch_create(int n_grids, fdtd_grid *const *grids, void *cuda_stream, fdtd_batch **out);

/* Queue n steps of every domain on the batch stream (asynchronous).  Each
 * grid's step count advances by n. */
int fdtd_batch_step(fdtd_batch *b, int n);

/* Wait for the batch stream; FDTD_ETIMEOUT if a bounded wait gave up. */
int fdtd_batch_synchronize(fdtd_batch *b);

/* Persistent CTAs and work items of launch 0 (planes between the z layers)
 * or 1 (z-layer planes). */
int fdtd_batch_launch_info(const fdtd_batch *b, int launch, int *ctas, int *items);

const char *fdtd_batch_last_error(const fdtd_batch *b);
void fdtd_batch_destroy(fdtd_batch *b);

/* Self-test of the bounded waits (a library addition).  Every wait of the
 * step kernel on an mbarrier gives up after 2 s, records the failure, drains
 * its copies in flight and returns, so that fdtd_synchronize() reports
 * FDTD_ETIMEOUT instead of the GPU hanging.  This call runs the same wait
 * routine on an mbarrier phase that nothing completes, with a limit of
 * `seconds` (0 < seconds <= 10), on cuda_stream, and synchronises it.
 * Returns FDTD_ETIMEOUT when the wait gave up as designed (the expected
 * result), FDTD_OK if it completed, FDTD_EINVAL for a bad limit,
 * FDTD_ECUDA on a CUDA error.  The context stays usable afterwards. */
int fdtd_selftest_wait(double seconds, void *cuda_stream);

/* Checkpoint / resume of a finalized grid (a library addition; the paper's
 * solver has no counterpart).  The state is everything the step reads that
 * changes while stepping: the six fields, the twelve CPML auxiliaries (when
 * the grid has a CPML), the Debye currents, the oblique-wire currents and
 * charges, the probe record [n_probes x probe_capacity] and the step count.  Stepping a grid after fdtd_load_state continues bit for bit
 * as the grid that saved the state did.
 *   fdtd_save_state: host_buf NULL -> *bytes = the size needed, FDTD_OK;
 *     otherwise *bytes is the buffer size on entry (FDTD_EINVAL, with the
 *     size needed in *bytes, when too small) and the bytes written on return.
 *     Synchronises the grid's stream.
 *   fdtd_load_state: the grid must have the same sizes, CPML thickness,
 *     probe count and probe capacity as the one that saved (FDTD_EINVAL
 *     otherwise, or for a buffer that is not a saved state).  Materials,
 *     wires and sources are the caller's to rebuild identically; they are
 *     not part of the state.  Synchronises the grid's stream. */
int fdtd_save_state(fdtd_grid *g, void *host_buf, size_t *bytes);
int fdtd_load_state(fdtd_grid *g, const void *host_buf, size_t bytes);

double fdtd_get_dt(const fdtd_grid *g);
long fdtd_get_step(const fdtd_grid *g);
int fdtd_num_classes(const fdtd_grid *g);
const char *fdtd_last_error(const fdtd_grid *g);
void fdtd_destroy(fdtd_grid *g);

#ifdef __cplusplus
}
#endif

#endif /* FDTD_GB300_FDTD_H */
