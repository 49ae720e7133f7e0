// stage_layout.cuh — shared-memory layout of the stage-sweep kernel (host and device).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "program.h"

namespace svk {

// per-group thread-offset table in shared memory only while it stays small
__host__ __device__ __forceinline__ bool group_table_fits(uint32_t n_groups, uint32_t nthr) {
    return (size_t)n_groups * nthr * 12 <= 24 * 1024;
}
// per-(phase slot, thread) thread-bit angle table, likewise
__host__ __device__ __forceinline__ bool angle_table_fits(uint32_t n_phase, uint32_t nthr, size_t angb) {
    return (size_t)n_phase * nthr * angb <= 16 * 1024;
}

// ---------------------------------------------------------------------------
// shared-memory layout of k_stage (identical on host and device)
// ---------------------------------------------------------------------------
struct SmemLayout {
    size_t groups, ops, slots, ang, gfix, chp, gsoff, chs, gsm, tang, total;
};
__host__ __device__ __forceinline__ size_t align_up(size_t x, size_t a) { return (x + a - 1) & ~(a - 1); }
__host__ __device__ __forceinline__ SmemLayout smem_layout(int elem_bytes, int nv, int nb, uint32_t T,
                                                           uint32_t n_groups, uint32_t n_ops, uint32_t n_phase,
                                                           uint32_t n_slots, uint32_t nthr, int nch) {
    const size_t opb = elem_bytes == 8 ? sizeof(DevOp<float>) : sizeof(DevOp<double>);
    const size_t slb = elem_bytes == 8 ? sizeof(PhaseSlot<float>) : sizeof(PhaseSlot<double>);
    const size_t angb = elem_bytes == 8 ? sizeof(uint32_t) : sizeof(double);
    const uint32_t ngt = group_table_fits(n_groups, nthr) ? n_groups : 0;
    SmemLayout L;
    size_t o = ((size_t)elem_bytes << T) * nb * nv;   // nv vectors x nb buffers
    L.groups = o;  o += n_groups * sizeof(Group);
    L.ops = o;     o += n_ops * opb;
    L.slots = o;   o += n_phase * slb;
    L.ang = o;     o = align_up(o + n_phase * angb, 16);
    L.gfix = o;    o += (size_t)ngt * nthr * 8;
    L.chp = o;     o += (size_t)nch * 8;
    L.gsoff = o;   o += (size_t)ngt * nthr * 4;
    L.chs = o;     o = align_up(o + (size_t)nch * 4, 16);
    L.gsm = o;     o = align_up(o + ((nv == 2) ? (size_t)n_slots * ((nthr + 31) / 32) * sizeof(double) : 0), 16);
    L.tang = o;    o += angle_table_fits(n_phase, nthr, angb) ? (size_t)n_phase * nthr * angb : 0;
    L.total = o;
    return L;
}

inline size_t smem_bytes_nb(int elem_bytes, const Stage& st, int nv, int nb) {
    const int R = (int)st.R;
    const int nch = (1 << R) / (16 / elem_bytes);
    return smem_layout(elem_bytes, nv, nb, st.T, st.n_groups, st.n_ops, st.n_phase, st.n_slots,
                       1u << (st.T - st.R), nch > 0 ? nch : 1).total;
}

}  // namespace svk
