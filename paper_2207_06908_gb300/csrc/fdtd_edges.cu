// fdtd_edges.cu -- the source/probe kernel: the ideal sources (Kuklin,
// arXiv 2207.06908, Sec. 2.1) and the probes of the Sec. 4 model files
// (fdtd_srcprobe.cuh), applied right after the step kernels (and, with Debye
// media, the dispersive-media kernel) of the same step.
// Oblique thin wires (Sec. 2.3, the Guiffaut formalism read in
// Holland-Simpson form): a separate kernel, concurrent with the step
// kernels, takes the segment currents to t_{n+1/2} from E^n gathered along
// each segment and the node potentials; this kernel, before the sources,
// adds those currents to E^{n+1} through the same edge shares and takes the
// node charges to t_{n+1}.
// One CTA per grid (one per domain in a batch, for the gather as well); a
// device-side step counter indexes the source samples and the probe slots,
// so the launches can be replayed inside a CUDA graph.
#include "fdtd_srcprobe.cuh"

namespace fdtd {
namespace {

constexpr int kWireSegShared = 4096;  // segment currents kept in shared memory for the scatter

// Oblique wires, first half of a step (all threads of the CTA): segment
// currents to t_{n+1/2} from E^n (the step's input, which the step kernels
// only read) and Q^n, so this runs concurrently with the step kernels.  Every
// sum has a fixed order, so a run repeats bit for bit.  The gather is
// flattened over (segment, edge) entries and staged in shared memory a
// chunk of whole segments at a time, so the loads of all threads are in
// flight together.
__device__ __forceinline__ void wire_gather_body(const EdgeArgs &a, long long n)
{
    const WireArgs &w = a.w;
    extern __shared__ float wire_smem[];
    float *prod = wire_smem;
    for (int c = 0; c < w.n_chunk; ++c) {
        // chunks of whole segments (host-built): segments own consecutive entry ranges
        const int lo = w.chunk[c], hi = w.chunk[c + 1];
        const int e_lo = w.seg[lo].e0;
        const int n_e = w.seg[hi - 1].e0 + w.seg[hi - 1].ne - e_lo;
#pragma unroll 4
        for (int q = threadIdx.x; q < n_e; q += blockDim.x) {
            const OEdge ed = w.edge[e_lo + q];
            prod[q] = in_bounds(ed.idx, a.plane * a.nz, 8, a.bounds) ? ed.wg * a.Ein[ed.comp][ed.idx] : 0.f;
        }
        __syncthreads();
        // L' dl dI/dt = E_s dl - (V_b - V_a) + EMF - R I, centred at t_n (the
        // R I term at the mean of the two half steps)
        for (int s = lo + threadIdx.x; s < hi; s += blockDim.x) {
            const OSeg sg = w.seg[s];
            float es = 0.f;
            for (int e = sg.e0 - e_lo; e < sg.e0 - e_lo + sg.ne; ++e) es += prod[e];
            const float va = w.node[sg.a].grounded ? 0.f : w.V[sg.a];
            const float vb = w.node[sg.b].grounded ? 0.f : w.V[sg.b];
            float inc = sg.cI * es - sg.cIV * (vb - va);
            for (int q = sg.s0; q < sg.s0 + sg.ns; ++q) {
                const OSrc sr = w.src[q];
                if (n < sr.n) inc += sr.cIV * w.samples[sr.off + n];
            }
            w.I[s] = sg.rk * w.I[s] + sg.rd * inc;
        }
        __syncthreads();
    }
}

// second half, after the step kernels: the segment currents in Ampere's law
// at t_{n+1/2} (four coupled edges per thread per pass, their field loads in
// flight together), then the node charges to t_{n+1}
__device__ __forceinline__ void wire_scatter_body(const EdgeArgs &a)
{
    const WireArgs &w = a.w;
    extern __shared__ float wire_smem[];
    float *Ish = wire_smem;
    for (int s = threadIdx.x; s < w.n_seg && s < kWireSegShared; s += blockDim.x) Ish[s] = w.I[s];
    __syncthreads();
    auto cur = [&](int s) { return s < kWireSegShared ? Ish[s] : w.I[s]; };
    for (int base = threadIdx.x; base < w.n_scat; base += 4 * blockDim.x) {
        OScat sc[4];
        float ev[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int u = base + k * blockDim.x;
            if (u < w.n_scat) {
                sc[k] = w.scat[u];
                if (!in_bounds(sc[k].idx, a.plane * a.nz, 9, a.bounds)) sc[k].idx = 0;   // bounds-checked build only
                ev[k] = a.E[sc[k].comp][sc[k].idx];
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (base + k * blockDim.x >= w.n_scat) break;
            float sum = 0.f;
            for (int t = sc[k].t0; t < sc[k].t0 + sc[k].nt; ++t) {
                const OTerm tm = w.term[t];
                sum += tm.ws * cur(tm.seg);
            }
            a.E[sc[k].comp][sc[k].idx] = ev[k] - sum;
        }
    }
    for (int m = threadIdx.x; m < w.n_node; m += blockDim.x) {
        const ONode nd = w.node[m];
        if (nd.grounded) {
            w.Q[m] = 0.f;
            w.V[m] = 0.f;
            continue;
        }
        float net = 0.f;
        for (int q = nd.adj0; q < nd.adj0 + nd.nadj; ++q) {
            const int t = w.adj[q];
            net += (t & 1) ? cur(t >> 1) : -cur(t >> 1);
        }
        // V^{n+1} from K Q^{n+1} = e0 V^{n+1} + sum_p P_p^{n+1}, the charge
        // and polarisation updates substituted
        float *P = w.P + (size_t)m * 4;
        const float V = w.V[m], Q = w.Q[m];
        float spb = 0.f, spa = 0.f;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            spb += nd.pb[p];
            spa += nd.pa[p] * P[p];
        }
        const float Vn = (nd.K * (Q + a.dt * net) - (nd.cs + spb) * V - spa) / (nd.e0 + spb + nd.cs);
#pragma unroll
        for (int p = 0; p < 4; ++p) P[p] = nd.pa[p] * P[p] + nd.pb[p] * (Vn + V);
        w.Q[m] = Q + a.dt * net - nd.cs / nd.K * (Vn + V);
        w.V[m] = Vn;
    }
    __syncthreads();
}

__device__ __forceinline__ void edge_body(const EdgeArgs &a)
{
    __shared__ long long n_s;
    if (threadIdx.x == 0) n_s = __ldcg(a.step) + a.step_t;
    __syncthreads();
    const long long n = n_s;
    if (a.w.n_seg > 0 && !a.wire_done) wire_scatter_body(a);
    src_probe_body(a, n);
}

__global__ void edge_kernel(const EdgeArgs a) { edge_body(a); }

__global__ void wire_finish_kernel(const EdgeArgs a) { wire_scatter_body(a); }

__global__ void wire_gather_kernel(const EdgeArgs a)
{
    __shared__ long long n_s;
    if (threadIdx.x == 0) n_s = *a.step + a.step_t;
    __syncthreads();
    wire_gather_body(a, n_s);
}

__global__ void edge_batch_kernel(const EdgeArgs *e, int parity)
{
    __shared__ EdgeArgs a;
    if (threadIdx.x == 0) a = e[2 * blockIdx.x + parity];
    __syncthreads();
    if (a.n_src > 0 || a.n_probes > 0 || a.w.n_seg > 0) edge_body(a);
}

// one CTA per domain of a batch: the oblique wires' first half of the step
__global__ void wire_gather_batch_kernel(const EdgeArgs *e, int parity)
{
    __shared__ EdgeArgs a;
    __shared__ long long n_s;
    if (threadIdx.x == 0) {
        a = e[2 * blockIdx.x + parity];
        if (a.w.n_seg > 0) n_s = __ldcg(a.step) + a.step_t;
    }
    __syncthreads();
    if (a.w.n_seg > 0) wire_gather_body(a, n_s);
}

}  // namespace

cudaError_t launch_edges(const EdgeArgs &a, cudaStream_t s)
{
    // oblique wires are latency-bound loops over their segments and edges:
    // a full CTA keeps enough loads in flight
    const bool wires = a.w.n_seg > 0;
    edge_kernel<<<1, wires ? 1024 : 128, wires ? kWireSegShared * sizeof(float) : 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_wire_finish(const EdgeArgs &a, cudaStream_t s)
{
    wire_finish_kernel<<<1, 1024, kWireSegShared * sizeof(float), s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_wire_gather(const EdgeArgs &a, cudaStream_t s)
{
    // latency-bound loops over segments and edges: a full CTA keeps enough
    // loads in flight
    wire_gather_kernel<<<1, 1024, kWireChunk * sizeof(float), s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_edges_batch(const EdgeArgs *e, int n_domains, int parity, bool wires, cudaStream_t s)
{
    if (wires) edge_batch_kernel<<<n_domains, 1024, kWireSegShared * sizeof(float), s>>>(e, parity);
    else edge_batch_kernel<<<n_domains, 128, 0, s>>>(e, parity);
    return cudaGetLastError();
}

cudaError_t launch_wire_gather_batch(const EdgeArgs *e, int n_domains, int parity, cudaStream_t s)
{
    wire_gather_batch_kernel<<<n_domains, 1024, kWireChunk * sizeof(float), s>>>(e, parity);
    return cudaGetLastError();
}

}  // namespace fdtd
