"""Regenerates the PacLayout table of tmop_pa_compact.cu (the padded strides
of the stage buffers of pac_kernel) by counting shared-memory bank conflicts.

Model: 32 banks of 4-byte words. A 4-byte warp access costs as many
wavefronts as the largest number of distinct words it puts on one bank; an
8-byte access is served by half warps, each costing the largest number of
distinct words on one bank among its 16 lanes' two words. Every access of
the stages is enumerated exactly as pac_fwd, pac_adj, the pointwise stage
and the gather/scatter staging issue it (lanes t = lane + 32 k over the
stage's rows), and each buffer's strides are chosen independently (no
instruction touches two buffers): lowest total wavefronts, ties to the
smallest buffer.

    python pac_layout_search.py        # prints one TMOP_PAC_LAYOUT line per (n, q)
"""
import itertools

PAIRS = [(2, 2), (2, 3), (3, 3), (3, 4), (4, 4), (4, 5), (5, 5), (5, 6)]
NC = 3


def wf32(addrs):
    banks = {}
    for a in addrs:
        banks.setdefault(a % 32, set()).add(a)
    return max(len(s) for s in banks.values()) if banks else 0


def wf64(addrs):
    total = 0
    for half in (addrs[:16], addrs[16:]):
        if not half:
            continue
        banks = {}
        for a in half:
            for w in (a, a + 1):
                banks.setdefault(w % 32, set()).add(w)
        total += max(len(s) for s in banks.values())
    return total


def cost(count, fns, wide):
    w = 0
    for base in range(0, count, 32):
        ts = range(base, min(base + 32, count))
        for fn in fns:
            a = [fn(t) for t in ts]
            w += wf64(a) if wide else wf32(a)
    return w


def search(N, Q1):
    NDOF, QP, QQ = N ** 3, Q1 ** 3, Q1 * Q1
    rows = lambda t: (t // (N * N), (t % (N * N)) // N, (t % (N * N)) % N)   # (c, l, j)
    f2 = lambda t: (t % Q1, (t // Q1) % N, t // (Q1 * N))                      # (q0, l, c)

    def cx(XR, XC):   # x / y: staging stores, stage-1 loads, last adjoint stores, scatter loads
        A = lambda c, lj, i: c * XC + lj * XR + i
        st = cost(NDOF, [lambda t, c=c: A(c, t // N, t % N) for c in range(3)], False)
        rw = cost(NC * N * N, [lambda t, i=i: A(t // (N * N), t % (N * N), i) for i in range(N)], False)
        return 2 * (st + rw)

    def ca(AR, AL, AC):   # stage-1 pairs
        A = lambda c, l, j, q0: c * AC + l * AL + j * AR + 2 * q0
        fa = [lambda t, q0=q0: A(*rows(t), q0) for q0 in range(Q1)]
        fb = [lambda t, j=j: A(f2(t)[2], f2(t)[1], j, f2(t)[0]) for j in range(N)]
        fs = [lambda t, j=j, k=k: A(f2(t)[2], f2(t)[1], j, f2(t)[0]) + k for j in range(N) for k in range(2)]
        return 2 * cost(NC * N * N, fa, True) + cost(NC * N * Q1, fb, True) + cost(NC * N * Q1, fs, False)

    def cbp(BQ, BL, BC):   # stage-2 pairs
        A = lambda c, l, q1, q0: c * BC + l * BL + q1 * BQ + 2 * q0
        rs = [lambda t, q1=q1, k=k: A(f2(t)[2], f2(t)[1], q1, f2(t)[0]) + k for q1 in range(Q1) for k in range(2)]
        rl = [lambda t, q1=q1: A(f2(t)[2], f2(t)[1], q1, f2(t)[0]) for q1 in range(Q1)]
        cl = [lambda t, l=l: A(t // QQ, l, (t % QQ) // Q1, t % Q1) for l in range(N)]
        cs = [lambda t, l=l, k=k: A(t // QQ, l, (t % QQ) // Q1, t % Q1) + k for l in range(N) for k in range(2)]
        return (cost(NC * N * Q1, rs, False) + cost(NC * N * Q1, rl, True) + cost(NC * QQ, cl, True)
                + cost(NC * QQ, cs, False))

    def cbs(SQ, SL, SC):   # stage-2 scalars
        A = lambda c, l, q1, q0: c * SC + l * SL + q1 * SQ + q0
        rs = [lambda t, q1=q1: A(f2(t)[2], f2(t)[1], q1, f2(t)[0]) for q1 in range(Q1)]
        cl = [lambda t, l=l: A(t // QQ, l, (t % QQ) // Q1, t % Q1) for l in range(N)]
        return 2 * cost(NC * N * Q1, rs, False) + 2 * cost(NC * QQ, cl, False)

    def cz(ZC, ZT):   # points: pairs (components 1, 2) and scalars (component 0)
        fp = [lambda t, q2=q2: (t // QQ) * ZC + 2 * (q2 * QQ + t % QQ) for q2 in range(Q1)]
        fs = [lambda t, q2=q2: (t // QQ) * ZT + q2 * QQ + t % QQ for q2 in range(Q1)]
        pp = [lambda t, c=c: c * ZC + 2 * t for c in range(3)]
        ps = [lambda t, c=c: c * ZT + t for c in range(3)]
        return 2 * (cost(NC * QQ, fp, True) + cost(NC * QQ, fs, False) + cost(QP, pp, True) + cost(QP, ps, False))

    def best(fn, cands):
        return min((fn(*c), c[-1], c) for c in cands)[2]

    X = best(cx, [(r, c) for r in range(N, N + 4) for c in range(N * N * r, N * N * r + 33)])
    A = best(ca, [(r, l, c) for r in range(2 * Q1, 2 * Q1 + 17, 2) for l in range(N * r, N * r + 33, 2)
                  for c in range(N * l, N * l + 65, 2)])
    Bp = best(cbp, [(q, l, c) for q in range(2 * Q1, 2 * Q1 + 17, 2) for l in range(Q1 * q, Q1 * q + 33, 2)
                    for c in range(N * l, N * l + 65, 2)])
    Bs = best(cbs, [(q, l, c) for q in range(Q1, Q1 + 3) for l in range(Q1 * q, Q1 * q + 12)
                    for c in range(N * l, N * l + 33)])
    Z = best(cz, [(zc, zt) for zc in range(2 * QP, 2 * QP + 65, 2) for zt in range(QP, QP + 33)])
    return X + A + Bp + Bs + Z


if __name__ == "__main__":
    for N, Q1 in PAIRS:
        vals = search(N, Q1)
        print("TMOP_PAC_LAYOUT(%s)" % ", ".join(str(v) for v in (N, Q1) + tuple(vals)), flush=True)
