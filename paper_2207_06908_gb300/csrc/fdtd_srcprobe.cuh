// fdtd_srcprobe.cuh -- the ideal sources of Kuklin, arXiv 2207.06908, Sec. 2.1
// (a current I on one edge, J = I / dx^2; a voltage held across one edge) and
// the probes of the Sec. 4 model files ("calculate": voltage = -sum E dl
// along a path, current = loop integral of H around an edge), applied to
// E^{n+1} once every kernel of step n that writes it has finished.
// Device code of the source/probe kernels (one grid, one CTA per domain of a
// batch).
#pragma once

#include "fdtd_internal.h"

namespace fdtd {
namespace {

__device__ __forceinline__ long long eidx(const EdgeArgs &a, int i, int j, int k)
{
    return (long long)k * a.plane + (long long)j * a.pitch + i;
}

// Sources, then probes, of step n, by all threads of one CTA; the fields are
// read through L2, where the step kernels' stores are.
// The descriptors of each thread's first source and probe are loaded before
// anything waits on them, so the chain of dependent loads is short.
__device__ __forceinline__ void src_probe_body(const EdgeArgs &a, long long n)
{
    const int t = threadIdx.x;
    SourceDesc sd0{};
    ProbeDesc pd0{};
    if (t < a.n_src) sd0 = a.src[t];
    if (t < a.n_probes) pd0 = a.probes[t];
    float I0 = 0.f;
    if (t < a.n_src && n < sd0.n_samples) I0 = __ldg(a.samples + sd0.sample_off + n);
    const int n_cur = a.skip_src ? 0 : a.n_src;     // current sources already applied by the step kernel
    for (int q = t; q < n_cur; q += blockDim.x) {
        const SourceDesc sd = q == t ? sd0 : a.src[q];
        if (sd.hard) continue;
        const float I = q == t ? I0 : (n < sd.n_samples ? __ldg(a.samples + sd.sample_off + n) : 0.f);
        const float add = sd.coef * I;
        if (!in_bounds(sd.idx, a.plane * a.nz, 6, a.bounds)) continue;
        atomicAdd(a.E[sd.comp] + sd.idx, add);
        // a dispersive edge: the currents already advanced with E^{n+1}
        // before the source; they take its share, be_p times the increment
        if (sd.jidx >= 0 && a.J)
#pragma unroll
            for (int p = 0; p < kMaxPoles; ++p)
                if (p < a.npoles && sd.be[p] != 0.f)
                    atomicAdd(a.J + (long long)(sd.comp * a.npoles + p) * a.jstride + sd.jidx, sd.be[p] * add);
    }
    __syncthreads();
    // ideal voltage sources, after the current sources: E^{n+1} = -V / dx
    // (and on a dispersive edge the currents take be_p times the change)
    for (int q = t; q < a.n_src; q += blockDim.x) {
        const SourceDesc sd = q == t ? sd0 : a.src[q];
        if (!sd.hard) continue;
        const float V = q == t ? I0 : (n < sd.n_samples ? __ldg(a.samples + sd.sample_off + n) : 0.f);
        if (!in_bounds(sd.idx, a.plane * a.nz, 6, a.bounds)) continue;
        float *e = a.E[sd.comp] + sd.idx;
        const float old = __ldcg(e), v = sd.vcoef * V;
        *e = v;
        if (sd.jidx >= 0 && a.J)
#pragma unroll
            for (int p = 0; p < kMaxPoles; ++p)
                if (p < a.npoles && sd.be[p] != 0.f)
                    atomicAdd(a.J + (long long)(sd.comp * a.npoles + p) * a.jstride + sd.jidx, sd.be[p] * (v - old));
    }
    __syncthreads();
    if (n < a.capacity) {
        for (int p = t; p < a.n_probes; p += blockDim.x) {
            const ProbeDesc pr = p == t ? pd0 : a.probes[p];
            float v = 0.f;
            if (pr.kind == 4) {
                v = __ldcg(a.w.I + pr.i);       // oblique-wire segment current
            } else if (pr.kind == 5) {
                v = __ldcg(a.w.V + pr.i);       // oblique-wire node: in-cell potential
            } else if (pr.kind == 2 || pr.kind == 3) {
                const long long o = eidx(a, pr.i, pr.j, pr.k);
                if (in_bounds(o, a.plane * a.nz, 7, a.bounds)) v = __ldcg((pr.kind == 2 ? a.E : a.H)[pr.axis] + o);
            } else if (pr.kind == 0) {
                // consecutive edges along the path's axis, summed in path order
                const float *Ep = a.E[pr.axis] + eidx(a, pr.i, pr.j, pr.k);
                const long long st = pr.axis == 0 ? 1 : (pr.axis == 1 ? (long long)a.pitch : a.plane);
#pragma unroll 4
                for (int e = 0; e < pr.n_edges; ++e)
                    if (in_bounds(eidx(a, pr.i, pr.j, pr.k) + e * st, a.plane * a.nz, 7, a.bounds))
                        v -= __ldcg(Ep + e * st) * a.dx;
            } else {
                const float *Hx = a.H[0], *Hy = a.H[1], *Hz = a.H[2];
                const int i = pr.i, j = pr.j, k = pr.k;
                // the loop reads the edge's cell and its neighbour below along the
                // two other axes (lowest: one row below for a z edge, one plane
                // below otherwise)
                const long long o = eidx(a, i, j, k), lo = o - (pr.axis == 2 ? (long long)a.pitch : a.plane);
                if (!in_bounds(o, a.plane * a.nz, 7, a.bounds) || !in_bounds(lo, a.plane * a.nz, 7, a.bounds))
                    continue;
                if (pr.axis == 2)
                    v = a.dx * ((__ldcg(Hy + eidx(a, i, j, k)) - __ldcg(Hy + eidx(a, i - 1, j, k))) -
                                (__ldcg(Hx + eidx(a, i, j, k)) - __ldcg(Hx + eidx(a, i, j - 1, k))));
                else if (pr.axis == 0)
                    v = a.dx * ((__ldcg(Hz + eidx(a, i, j, k)) - __ldcg(Hz + eidx(a, i, j - 1, k))) -
                                (__ldcg(Hy + eidx(a, i, j, k)) - __ldcg(Hy + eidx(a, i, j, k - 1))));
                else
                    v = a.dx * ((__ldcg(Hx + eidx(a, i, j, k)) - __ldcg(Hx + eidx(a, i, j, k - 1))) -
                                (__ldcg(Hz + eidx(a, i, j, k)) - __ldcg(Hz + eidx(a, i - 1, j, k))));
            }
            a.probe_out[(long long)p * a.capacity + n] = v;
        }
    }
    __syncthreads();
    if (t == 0 && a.advance) *a.step = n + 1;
}

}  // namespace
}  // namespace fdtd
