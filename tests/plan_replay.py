"""Replays a library plan on the CPU with numpy, following the exact records the
kernels receive (initial-tensor recipes, step stride runs, arena offsets, scaling).

Test infrastructure only: it checks the host planner's bookkeeping without a GPU.
"""
import ctypes as C
import math

import numpy as np

MAXRUNS = 20


class Recipe(C.Structure):
    _fields_ = [("kind", C.c_int32), ("rank", C.c_int32), ("slot0", C.c_int32),
                ("nslot", C.c_int32), ("elems", C.c_int64), ("offset", C.c_int64),
                ("meta", C.c_int32), ("exp2", C.c_int32)]


class Slot(C.Structure):
    _fields_ = [("dimpos", C.c_int32), ("slice_ord", C.c_int32), ("absorbed", C.c_int32),
                ("pad", C.c_int32), ("dre", C.c_double), ("dim", C.c_double),
                ("ore", C.c_double), ("oim", C.c_double)]


class GradLeaf(C.Structure):
    _fields_ = [("meta", C.c_int32), ("rank", C.c_int32), ("slice_ord", C.c_int32 * 2),
                ("offset", C.c_int64), ("stride", C.c_int64 * 2)]


class Run(C.Structure):
    _fields_ = [("size", C.c_int64), ("sa", C.c_int64), ("sb", C.c_int64)]


class Run4(C.Structure):
    _fields_ = [("size", C.c_int64), ("sa", C.c_int64), ("sb", C.c_int64), ("sc", C.c_int64)]


class ConvRec(C.Structure):
    _fields_ = [("src_off", C.c_int64), ("dst_off", C.c_int64), ("elems", C.c_int64),
                ("src_meta", C.c_int32), ("dst_meta", C.c_int32)]


class TailStep(C.Structure):
    _fields_ = [("step", C.c_int32), ("meta_a", C.c_int32), ("meta_b", C.c_int32),
                ("pad", C.c_int32), ("off_a", C.c_int64), ("off_b", C.c_int64),
                ("off_c", C.c_int64)]


class Step(C.Structure):
    _fields_ = [("a", C.c_int32), ("b", C.c_int32), ("c", C.c_int32), ("kernel", C.c_int32),
                ("off_a", C.c_int64), ("off_b", C.c_int64), ("off_c", C.c_int64),
                ("R", C.c_int64), ("K", C.c_int64), ("N", C.c_int64),
                ("nrow", C.c_int32), ("nk", C.c_int32), ("nn", C.c_int32),
                ("row", Run * MAXRUNS), ("kr", Run * MAXRUNS), ("nr", Run * MAXRUNS),
                ("rank_c", C.c_int32), ("chunks", C.c_int32),
                ("Bsz", C.c_int64), ("M", C.c_int64), ("ngb", C.c_int32), ("ngm", C.c_int32),
                ("ngn", C.c_int32), ("a_kinner", C.c_int32), ("b_kinner", C.c_int32),
                ("tc", C.c_int32), ("gb", Run4 * MAXRUNS), ("gm", Run4 * MAXRUNS),
                ("gn", Run4 * MAXRUNS)]


def _offsets(n, runs, nruns):
    """Per linear index x < n: (sum digit*sa, sum digit*sb) over the stride runs."""
    x = np.arange(n, dtype=np.int64)
    oa = np.zeros(n, dtype=np.int64)
    ob = np.zeros(n, dtype=np.int64)
    for i in range(nruns):
        sz = runs[i].size
        d = x % sz
        x = x // sz
        oa += d * runs[i].sa
        ob += d * runs[i].sb
    return oa, ob


def _offsets4(n, runs, nruns):
    x = np.arange(n, dtype=np.int64)
    o = [np.zeros(n, dtype=np.int64) for _ in range(3)]
    for i in range(nruns):
        sz = runs[i].size
        d = x % sz
        x = x // sz
        o[0] += d * runs[i].sa
        o[1] += d * runs[i].sb
        o[2] += d * runs[i].sc
    return o


def _gemm_view(st, arena, scale):
    """The step through its GEMM-view records (batch / m / n runs with C strides)."""
    ab, bb, cb = _offsets4(st.Bsz, st.gb, st.ngb)
    am, _, cm = _offsets4(st.M, st.gm, st.ngm)
    _, bn, cn = _offsets4(st.N, st.gn, st.ngn)
    ka, kb = _offsets(st.K, st.kr, st.nk)
    A = arena[st.off_a + ab[:, None, None] + am[None, :, None] + ka[None, None, :]]
    B = arena[st.off_b + bb[:, None, None] + kb[None, :, None] + bn[None, None, :]]
    Cv = np.einsum("bmk,bkn->bmn", A, B) * scale
    idx = st.off_c + cb[:, None, None] + cm[None, :, None] + cn[None, None, :]
    assert len(np.unique(idx)) == idx.size == st.R * st.N
    return idx, Cv


def replay(plan, split=False):
    sc = np.frombuffer(plan.debug_blob(3), dtype=np.int64)
    q, n_init, n_steps, n_slices, n_sliced, final_t, off_rec, off_slots, n_slots, step_sz = \
        [int(v) for v in sc[:10]]
    tail_first, n_tail, n_conv, off_conv, final_tail_off = [int(v) for v in sc[10:15]]
    assert step_sz == C.sizeof(Step), (step_sz, C.sizeof(Step))
    prog = plan.debug_blob(0)
    recs = [Recipe.from_buffer_copy(prog, off_rec + i * C.sizeof(Recipe)) for i in range(n_init)]
    slots = [Slot.from_buffer_copy(prog, off_slots + i * C.sizeof(Slot)) for i in range(n_slots)]
    sb = plan.debug_blob(1)
    steps = [Step.from_buffer_copy(sb, i * C.sizeof(Step)) for i in range(n_steps)]
    tinfo = np.frombuffer(plan.debug_blob(2), dtype=np.int64).reshape(-1, 2)
    fre, fim, fexp = np.frombuffer(plan.debug_blob(4), dtype=np.float64)
    arena_n = int((tinfo[:, 0] + tinfo[:, 1]).max())
    convs = [ConvRec.from_buffer_copy(prog, off_conv + i * C.sizeof(ConvRec)) for i in range(n_conv)]
    tb = plan.debug_blob(5)
    tails = [TailStep.from_buffer_copy(tb, i * C.sizeof(TailStep)) for i in range(n_tail)]
    tail_n = max([cr.dst_off + cr.elems for cr in convs] +
                 [ts.off_c + int(tinfo[steps[ts.step].c, 1]) for ts in tails] + [1])
    total = []
    for sl in range(n_slices):
        sdig = []
        s = sl
        for _ in range(n_sliced):
            sdig.append(s % q)
            s //= q
        arena = np.full(arena_n, np.nan + 0j, dtype=np.complex128)
        mx = {}
        ex = {}
        _build(recs, slots, q, sdig, arena, mx, ex)
        if split and n_tail > 0:
            # complex128 tail: widen the bulk tensors it reads, run its steps in the
            # tail region with the tail records' offsets and bookkeeping slots
            tail_region = np.full(max(1, tail_n), np.nan + 0j, dtype=np.complex128)
            for st in steps[:tail_first]:
                _step(st, arena, arena, mx, ex)
            for cr in convs:
                tail_region[cr.dst_off:cr.dst_off + cr.elems] = arena[cr.src_off:cr.src_off + cr.elems]
                mx[cr.dst_meta], ex[cr.dst_meta] = mx[cr.src_meta], ex[cr.src_meta]
            for ts in tails:
                st = Step.from_buffer_copy(bytes(steps[ts.step]))
                st.a, st.b = ts.meta_a, ts.meta_b
                st.off_a, st.off_b, st.off_c = ts.off_a, ts.off_b, ts.off_c
                _step(st, tail_region, tail_region, mx, ex)
            v = tail_region[final_tail_off]
            total.append((complex(v), ex[final_t]))
            continue
        for st in steps:
            _step(st, arena, arena, mx, ex)
        v = arena[tinfo[final_t, 0]]
        total.append((complex(v), ex[final_t]))
    # sum of slices, then the constant factor
    emax = max((e + math.frexp(abs(v))[1] for v, e in total if v != 0), default=0)
    z = sum(v * 2.0 ** (e - emax) for v, e in total)
    return complex(z) * complex(fre, fim), emax + int(fexp)


def _step(st, arena, out, mx, ex):
    """One step exactly as the kernels address it (operands and output in `arena`)."""
    oa, ob = _offsets(st.R, st.row, st.nrow)
    ka, kb = _offsets(st.K, st.kr, st.nk)
    _, nb = _offsets(st.N, st.nr, st.nn)
    A = arena[st.off_a + oa[:, None] + ka[None, :]]                 # R x K
    ea = math.frexp(mx[st.a])[1] if mx[st.a] > 0 else 0
    if st.b >= 0:
        B = arena[st.off_b + ob[:, None, None] + kb[None, :, None] + nb[None, None, :]]
        eb = math.frexp(mx[st.b])[1] if mx[st.b] > 0 else 0
        Cv = np.einsum("rk,rkn->nr", A, B)
        xb = ex[st.b]
    else:
        eb, xb = 0, 0
        Cv = A.sum(axis=1)[None, :]
    Cv = Cv * 2.0 ** -(ea + eb)
    flat = Cv.reshape(-1)   # C[n * R + r]
    if st.b >= 0:
        # the GEMM view of the same step must address the same entries
        idx, Cg = _gemm_view(st, arena, 2.0 ** -(ea + eb))
        ref = np.empty_like(flat)
        ref[idx.reshape(-1) - st.off_c] = Cg.reshape(-1)
        assert np.allclose(ref, flat, rtol=1e-12, atol=1e-300)
    out[st.off_c:st.off_c + flat.size] = flat
    assert not np.isnan(flat).any()
    mx[st.c] = float(np.max(np.maximum(np.abs(flat.real), np.abs(flat.imag))))
    ex[st.c] = ex[st.a] + xb + ea + eb


def _build(recs, slots, q, sdig, arena, mx, ex):
    """Initial tensors from their recipes, as k_build forms them."""
    for r in recs:
        e = np.arange(r.elems, dtype=np.int64)
        if r.kind == 1:
            val = np.ones(r.elems, dtype=np.complex128)
        else:
            val = np.zeros(r.elems, dtype=np.complex128)
            for s in range(q):
                prod = np.ones(r.elems, dtype=np.complex128)
                for j in range(r.nslot):
                    sl_ = slots[r.slot0 + j]
                    x = (e // q ** sl_.dimpos) % q if sl_.dimpos >= 0 else \
                        np.full(r.elems, sdig[sl_.slice_ord])
                    if sl_.absorbed:
                        prod = np.where(x == s, prod * complex(sl_.dre, sl_.dim),
                                        prod * complex(sl_.ore, sl_.oim))
                    else:
                        prod = np.where(x == s, prod, 0)
                val += prod
        arena[r.offset:r.offset + r.elems] = val
        mx[r.meta] = float(np.max(np.maximum(np.abs(val.real), np.abs(val.imag))))
        ex[r.meta] = r.exp2


def replay_grad(plan):
    """The reverse-pass program of a grad plan on the CPU: returns (Z as (mantissa,
    exponent), accumulators (groups, q*q) complex, their exponents), as pk_grad's
    kernels leave them for the host's last stage."""
    sc = np.frombuffer(plan.debug_blob(7), dtype=np.int64)
    (n_steps, n_meta, arena_n, root_off, root_meta, off_rec, off_slots, off_leaves, n_leaves,
     n_slices, leaf_sz, n_init, n_slots, q, n_sliced, slot_sz) = [int(v) for v in sc[:16]]
    assert leaf_sz == C.sizeof(GradLeaf) and slot_sz == C.sizeof(Slot)
    prog = plan.debug_blob(8)
    recs = [Recipe.from_buffer_copy(prog, off_rec + i * C.sizeof(Recipe)) for i in range(n_init)]
    slots = [Slot.from_buffer_copy(prog, off_slots + i * C.sizeof(Slot)) for i in range(n_slots)]
    leaves = [GradLeaf.from_buffer_copy(prog, off_leaves + i * C.sizeof(GradLeaf))
              for i in range(n_leaves)]
    sb = plan.debug_blob(6)
    steps = [Step.from_buffer_copy(sb, i * C.sizeof(Step)) for i in range(n_steps)]
    acc = np.zeros((max(1, n_leaves), q * q), dtype=np.complex128)
    acc_exp = np.zeros(max(1, n_leaves), dtype=np.int64)
    total = []
    for sl in range(n_slices):
        sdig = []
        s = sl
        for _ in range(n_sliced):
            sdig.append(s % q)
            s //= q
        arena = np.full(max(1, arena_n), np.nan + 0j, dtype=np.complex128)
        mx, ex = {}, {}
        _build(recs, slots, q, sdig, arena, mx, ex)
        for st in steps:
            _step(st, arena, arena, mx, ex)
        total.append((complex(arena[root_off]), ex[root_meta]))
        for g, L in enumerate(leaves):
            n = q * q if L.rank == 2 else q
            inc = np.zeros(n, dtype=np.complex128)
            for e in range(n):
                d = (e // q, e % q) if L.rank == 2 else (e, 0)
                off, skip = 0, False
                for j in range(L.rank):
                    if L.slice_ord[j] >= 0:
                        skip |= d[j] != sdig[L.slice_ord[j]]
                    else:
                        off += d[j] * L.stride[j]
                if not skip:
                    inc[e] = 1.0 if L.meta < 0 else arena[L.offset + off]
            ev = 0 if L.meta < 0 else ex[L.meta]
            mi = float(np.max(np.maximum(np.abs(inc.real), np.abs(inc.imag))))
            ma = float(np.max(np.maximum(np.abs(acc[g, :n].real), np.abs(acc[g, :n].imag))))
            if mi == 0:
                continue
            enew = ev + math.frexp(mi)[1]
            if ma > 0:
                enew = max(enew, int(acc_exp[g]) + math.frexp(ma)[1])
            so = 2.0 ** (int(acc_exp[g]) - enew) if ma > 0 else 0.0
            acc[g, :n] = acc[g, :n] * so + inc * 2.0 ** (ev - enew)
            acc_exp[g] = enew
    emax = max((e + math.frexp(abs(v))[1] for v, e in total if v != 0), default=0)
    z = sum(v * 2.0 ** (e - emax) for v, e in total)
    return (complex(z), emax), acc[:n_leaves], acc_exp[:n_leaves]


def _ring_mul(x, y, p, qm2):
    """(a + b t)(c + d t) in F_p[t]/(t^2 - (q-2) t + 1), elementwise on int64 arrays."""
    a, b = x
    c, d = y
    ac, bd = (a * c) % p, (b * d) % p
    cross = ((a * d) % p + (b * c) % p) % p
    return (ac - bd) % p, (cross + (qm2 * bd) % p) % p


def _tpow(n, p, qm2):
    """t^n as a pair of ints (t^-1 = (q-2) - t)."""
    base = (0, 1) if n >= 0 else (qm2, p - 1)
    res = (1, 0)
    m = abs(n)
    while m:
        if m & 1:
            res = tuple(int(v) for v in _ring_mul(res, base, p, qm2))
        base = tuple(int(v) for v in _ring_mul(base, base, p, qm2))
        m >>= 1
    return res


def replay_exact(plan, p):
    """Z(q) mod p as (a, b), Z = a + b t, following the records the exact kernels read:
    recipes with the packed exact clause data (Slot.pad: mult, signsum), every step
    through its stride runs, the slices, then the folded loops' factor."""
    sc = np.frombuffer(plan.debug_blob(3), dtype=np.int64)
    q, n_init, n_steps, n_slices, n_sliced, final_t, off_rec, off_slots, n_slots, step_sz = \
        [int(v) for v in sc[:10]]
    loop_count, loop_sign = int(sc[15]), int(sc[16])
    prog = plan.debug_blob(0)
    recs = [Recipe.from_buffer_copy(prog, off_rec + i * C.sizeof(Recipe)) for i in range(n_init)]
    slots = [Slot.from_buffer_copy(prog, off_slots + i * C.sizeof(Slot)) for i in range(n_slots)]
    sb = plan.debug_blob(1)
    steps = [Step.from_buffer_copy(sb, i * C.sizeof(Step)) for i in range(n_steps)]
    tinfo = np.frombuffer(plan.debug_blob(2), dtype=np.int64).reshape(-1, 2)
    arena_n = int((tinfo[:, 0] + tinfo[:, 1]).max())
    qm2 = (q - 2) % p
    total = (0, 0)
    for sl in range(n_slices):
        sdig, s = [], sl
        for _ in range(n_sliced):
            sdig.append(s % q)
            s //= q
        A_ = np.zeros(arena_n, dtype=np.int64)
        B_ = np.zeros(arena_n, dtype=np.int64)
        for r in recs:
            e = np.arange(r.elems, dtype=np.int64)
            if r.kind == 1:
                va, vb = np.ones(r.elems, dtype=np.int64), np.zeros(r.elems, dtype=np.int64)
            else:
                va, vb = np.zeros(r.elems, dtype=np.int64), np.zeros(r.elems, dtype=np.int64)
                for spin in range(q):
                    pa, pb = np.ones(r.elems, dtype=np.int64), np.zeros(r.elems, dtype=np.int64)
                    for j in range(r.nslot):
                        sl_ = slots[r.slot0 + j]
                        x = (e // q ** sl_.dimpos) % q if sl_.dimpos >= 0 else \
                            np.full(r.elems, sdig[sl_.slice_ord])
                        if sl_.absorbed:
                            mult = sl_.pad & 0xFFFF
                            sign = ((sl_.pad >> 16) & 0xFFFF)
                            sign = sign - 0x10000 if sign >= 0x8000 else sign
                            dg = _tpow(-sign, p, qm2)
                            if mult & 1:
                                dg = ((-dg[0]) % p, (-dg[1]) % p)
                            na, nb = _ring_mul((pa, pb), (np.int64(dg[0]), np.int64(dg[1])), p, qm2)
                            pa, pb = np.where(x == spin, na, pa), np.where(x == spin, nb, pb)
                        else:
                            pa, pb = np.where(x == spin, pa, 0), np.where(x == spin, pb, 0)
                    va, vb = (va + pa) % p, (vb + pb) % p
            A_[r.offset:r.offset + r.elems] = va
            B_[r.offset:r.offset + r.elems] = vb
        for st in steps:
            oa, ob = _offsets(st.R, st.row, st.nrow)
            ka, kb = _offsets(st.K, st.kr, st.nk)
            _, nb = _offsets(st.N, st.nr, st.nn)
            ca = np.zeros((st.N, st.R), dtype=np.int64)
            cb = np.zeros((st.N, st.R), dtype=np.int64)
            for k in range(st.K):
                ia = st.off_a + oa + ka[k]
                xa, xb = A_[ia][None, :], B_[ia][None, :]
                if st.b >= 0:
                    ib = st.off_b + ob[None, :] + kb[k] + nb[:, None]
                    pa, pb = _ring_mul((xa, xb), (A_[ib], B_[ib]), p, qm2)
                else:
                    pa, pb = xa, xb
                ca, cb = (ca + pa) % p, (cb + pb) % p
            A_[st.off_c:st.off_c + st.N * st.R] = ca.reshape(-1)
            B_[st.off_c:st.off_c + st.N * st.R] = cb.reshape(-1)
        off = int(tinfo[final_t, 0])
        total = ((total[0] + int(A_[off])) % p, (total[1] + int(B_[off])) % p)
    f = _tpow(-loop_sign, p, qm2)
    if loop_count & 1:
        f = ((-f[0]) % p, (-f[1]) % p)
    z = _ring_mul((np.int64(total[0]), np.int64(total[1])), (np.int64(f[0]), np.int64(f[1])), p, qm2)
    return int(z[0]), int(z[1])
