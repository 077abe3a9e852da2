// Step schedule of the dense apply (Algorithm 6 over Algorithm 4, one front or
// Section 4.2's two fronts): which quasi-1D solve a step of the persistent
// launch carries, and on which clusters.  Plain integer code, shared by the
// kernel and by the host-side schedule test; included inside dense.cu's
// anonymous namespace.
#pragma once

// Position j (0 .. 2B-2) of a block sweep (Algorithm 4 or 6) with centre block
// c: the forward pass visits the lower front upward (blocks 0..c-1), the upper
// front downward (B-1..c+1), then the centre; the backward pass the lower front
// downward (c-1..0), then the upper front upward (c+1..B-1).  One front: c = B-1.
enum { ROLE_L = 0, ROLE_U = 1, ROLE_C = 2 };
struct PassPos {
    int M, bwd, role;
};
__host__ __device__ __forceinline__ PassPos pass_pos(int j, int B, int c) {
    PassPos r;
    if (j < c) { r.M = j; r.bwd = 0; r.role = ROLE_L; }
    else if (j < B - 1) { r.M = B - 1 - (j - c); r.bwd = 0; r.role = ROLE_U; }
    else if (j == B - 1) { r.M = c; r.bwd = 0; r.role = ROLE_C; }
    else if (j < B + c) { r.M = c - 1 - (j - B); r.bwd = 1; r.role = ROLE_L; }
    else { r.M = c + 1 + (j - B - c); r.bwd = 1; r.role = ROLE_U; }
    return r;
}

// Operator slot of a solve within its slab's table: line blocks 0..B-1 (one
// operator serves both passes, except at the boundary blocks), B: the backward
// map of block 0, B+1: the backward map of block B-1 (two fronts only).  The
// global index of slot q of slab M: M*B + q, B*B + M, or B*B + B + M.
__host__ __device__ __forceinline__ int op_slot(int Mp, int bwd, int B) {
    return !bwd ? Mp : (Mp == 0 ? B : (Mp == B - 1 ? B + 1 : Mp));
}
__host__ __device__ __forceinline__ int op_index(int M, int slot, int B) {
    return slot < B ? M * B + slot : (slot == B ? B * B + M : B * B + B + M);
}
__host__ __device__ __forceinline__ int dense_nops(int B) { return B * B + 2 * B; }

// The problem / operator index of solve s of a full apply, and its roles.
struct OpInfo {
    int M, Mp, od, id, p;   // slab, line block, outer / inner direction (0 fwd, 1 bwd), operator
    int rz, ry;             // roles of the slab and the line block (ROLE_*)
};
__host__ __device__ __forceinline__ OpInfo op_info(int s, int B, int c, int two) {
    const int per = 2 * B - 1;
    const int jo = s / per, ji = s - jo * per;
    OpInfo o;
    if (!two) {
        // one front (c = B-1): the closed form of pass_pos, cheaper on the step's critical path
        o.od = jo >= B;
        o.M = o.od ? 2 * B - 2 - jo : jo;
        o.rz = (!o.od && o.M == B - 1) ? ROLE_C : ROLE_L;
        o.id = ji >= B;
        o.Mp = o.id ? 2 * B - 2 - ji : ji;
        o.ry = (!o.id && o.Mp == B - 1) ? ROLE_C : ROLE_L;
        o.p = (o.Mp > 0) ? o.M * B + o.Mp : (o.id == 0 ? o.M * B : B * B + o.M);
        return o;
    }
    const PassPos po = pass_pos(jo, B, c), pi = pass_pos(ji, B, c);
    o.M = po.M;
    o.od = po.bwd;
    o.rz = po.role;
    o.Mp = pi.M;
    o.id = pi.bwd;
    o.ry = pi.role;
    o.p = op_index(o.M, op_slot(o.Mp, o.id, B), B);
    return o;
}

// Inner steps of one slab visit.  One front: the 2B-1 solves of Algorithm 4 one
// after the other.  Two fronts: the lower and the upper front are independent,
// so they run side by side on two groups of clusters: forward step t solves the
// lower front's block t and the upper front's block B - t (the upper front one
// step behind, so that the two never couple into the centre line in the same
// step), then the centre, then backward step u solves blocks c-1-u and c+1+u.
__host__ __device__ __forceinline__ int inner_steps(int B, int c, int two) {
    if (!two) return 2 * B - 1;
    const int Lc = c, Uc = B - 1 - c;
    return (Lc > Uc + 1 ? Lc : Uc + 1) + 1 + (Lc > Uc ? Lc : Uc);
}

// Step s of a launch: slab visit jo = s / spv (Algorithm 6's order, spv = 1 +
// inner steps), then k = s % spv: k = 0 is the visit's boundary phase (write the
// previous visit's result to z, form this visit's right-hand side), k >= 1 is
// inner step k-1.  The last step is the final boundary phase.  With two fronts
// a step may hold two solves: clusters [0, ceil(nclus/2)) take the lower front's,
// the others the upper front's; mcid / mncl are this cluster's index among the
// clusters of its solve and their number.
struct StepInfo {
    int phase, jo, k;
    OpInfo o;
    int mcid, mncl;
};
__host__ __device__ __forceinline__ StepInfo step_info(int s, int B, int c, int two, int cid, int nclus) {
    StepInfo t;
    const int spv = inner_steps(B, c, two) + 1;
    t.jo = s / spv;
    t.k = s - t.jo * spv;
    t.phase = (t.k == 0);
    t.mcid = cid;
    t.mncl = nclus;
    if (t.phase) {
        t.o = OpInfo{0, 0, 0, 0, 0, 0, 0};
        return t;
    }
    if (!two) {
        t.o = op_info(t.jo * (2 * B - 1) + (t.k - 1), B, c, 0);
        return t;
    }
    const PassPos po = pass_pos(t.jo, B, c);
    const int tt = t.k - 1, Lc = c, Uc = B - 1 - c;
    const int F = Lc > Uc + 1 ? Lc : Uc + 1;
    int na = -1, nb = -1, bwd = 0, centre = 0;
    if (tt < F) {
        if (tt < Lc) na = tt;
        if (tt >= 1 && tt <= Uc) nb = B - tt;
    } else if (tt == F) {
        na = c;
        centre = 1;
    } else {
        const int u = tt - F - 1;
        if (u < Lc) na = c - 1 - u;
        if (u < Uc) nb = c + 1 + u;
        bwd = 1;
    }
    const int ncA = (nclus + 1) / 2;
    const bool both = na >= 0 && nb >= 0;
    const bool useB = nb >= 0 && (na < 0 || cid >= ncA);
    if (both) {
        t.mcid = useB ? cid - ncA : cid;
        t.mncl = useB ? nclus - ncA : ncA;
    }
    OpInfo o;
    o.M = po.M;
    o.od = po.bwd;
    o.rz = po.role;
    o.Mp = useB ? nb : na;
    o.id = bwd;
    o.ry = useB ? ROLE_U : (centre ? ROLE_C : ROLE_L);
    o.p = op_index(o.M, op_slot(o.Mp, o.id, B), B);
    t.o = o;
    return t;
}
