"""Learned initial iterate for TMOP Newton on 2D structured order-k meshes.

Pipeline (all arithmetic in libtmop_gb300.so; this module only sequences
calls and marshals arguments):

1. data:  many seeded jittered meshes are solved by plain Newton (Section 3.4
   line search, MINRES) as ONE problem -- the meshes are disjoint, so the
   Hessian is block diagonal and every block converges to its own minimiser;
   features are the 3x3-element patches of the jittered meshes, targets the
   Newton displacement of each centre element's owned nodes
   (tmop_patch_features / tmop_patch_targets).
2. train: MLP n_in -> 256 -> 256 -> 2k^2 on the GPU with the library's
   bfloat16 tensor-core forward/backward kernels and Adam.
3. propose: features of a new mesh -> MLP -> x0 + h * displacement at every
   free owned node (tmop_patch_apply). The proposal is kept only if it is
   valid (min det A > 0) and lowers F; otherwise Newton starts from x0.

With coarse=True (for domains whose optimum is not locally determined, such
as the curved-boundary workload) every step starts instead from the coarse
stage: the TMOP problem of the element-vertex grid (order 1) is solved by
Newton, its vertex displacement interpolated to the fine nodes
(tmop_lattice_vertices / tmop_lattice_prolong_add), and the network learns
and predicts only the residual from there.
"""
from __future__ import annotations

import ctypes as C
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import meshgen as mg
from . import tmop as tm

_MLP_SIGS = {
    "tmop_patch_features": ([C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int,
                             C.c_void_p], C.c_int),
    "tmop_patch_targets": ([C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p,
                            C.c_int, C.c_void_p], C.c_int),
    "tmop_patch_apply": ([C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int,
                          C.c_double, C.c_void_p, C.c_void_p], C.c_int),
    "tmop_lattice_vertices": ([C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p],
                              C.c_int),
    "tmop_lattice_prolong_add": ([C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                  C.c_int, C.c_void_p, C.c_void_p], C.c_int),
    "tmop_mlp_create": ([C.c_int, C.c_int, C.c_int, C.c_uint64, C.POINTER(C.c_void_p)], C.c_int),
    "tmop_mlp_destroy": ([C.c_void_p], None),
    "tmop_mlp_input_ld": ([C.c_void_p], C.c_int),
    "tmop_mlp_forward": ([C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p], C.c_int),
    "tmop_mlp_gradients": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p], C.c_int),
    "tmop_mlp_adam": ([C.c_void_p, C.c_float, C.c_void_p], C.c_int),
    "tmop_mlp_check": ([C.c_void_p, C.c_void_p], C.c_int),
    "tmop_mlp_num_params": ([C.c_void_p], C.c_size_t),
    "tmop_mlp_get": ([C.c_void_p, C.c_int, C.c_void_p, C.c_size_t], C.c_int),
    "tmop_mlp_set": ([C.c_void_p, C.c_void_p, C.c_size_t], C.c_int),
}
_loaded = False


def lib():
    global _loaded
    L = tm.load()
    if not _loaded:
        for name, (args, res) in _MLP_SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _loaded = True
    return L


def _check(rc, what):
    if rc != tm.OK:
        raise tm.TmopError(rc, what)


def _p(t):
    return C.c_void_p(t.data_ptr())


def _s():
    return tm._stream()


def n_features(order: int) -> int:
    return 2 * (3 * order + 1) ** 2


def n_targets(order: int) -> int:
    return 2 * order * order


class MLP:
    """The proposal network (wraps tmop_mlp_*)."""

    def __init__(self, n_in: int, n_out: int, hidden: int = 256, seed: int = 0):
        h = C.c_void_p()
        _check(lib().tmop_mlp_create(n_in, hidden, n_out, seed, C.byref(h)), "tmop_mlp_create")
        self._h, self.n_in, self.n_out, self.hidden = h, n_in, n_out, hidden
        self.ld = lib().tmop_mlp_input_ld(h)

    def close(self):
        if getattr(self, "_h", None):
            lib().tmop_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_params(self):
        return lib().tmop_mlp_num_params(self._h)

    def get(self, which=0) -> np.ndarray:
        out = np.zeros(self.num_params, dtype=np.float32)
        _check(lib().tmop_mlp_get(self._h, which, out.ctypes.data, out.size), "tmop_mlp_get")
        return out

    def set(self, flat: np.ndarray):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        _check(lib().tmop_mlp_set(self._h, flat.ctypes.data, flat.size), "tmop_mlp_set")

    def unflatten(self, flat):
        h, i, o = self.hidden, self.n_in, self.n_out
        sizes = [(h, i), (h,), (h, h), (h,), (o, h), (o,)]
        out, k = [], 0
        for s in sizes:
            n = int(np.prod(s))
            out.append(np.asarray(flat[k:k + n], dtype=np.float64).reshape(s))
            k += n
        return out

    def forward(self, X, Y=None):
        import torch
        B = X.shape[0]
        Y = torch.empty((B, 64), dtype=torch.float32, device=X.device) if Y is None else Y
        _check(lib().tmop_mlp_forward(self._h, _p(X), B, _p(Y), Y.shape[1], _s()), "tmop_mlp_forward")
        return Y

    def gradients(self, X, T, loss=None):
        _check(lib().tmop_mlp_gradients(self._h, _p(X), _p(T), T.shape[1], X.shape[0],
                                        None if loss is None else _p(loss), _s()), "tmop_mlp_gradients")

    def adam(self, lr: float):
        _check(lib().tmop_mlp_adam(self._h, lr, _s()), "tmop_mlp_adam")

    def check(self):
        """Raise if some GEMM since the last check gave up its bounded wait."""
        _check(lib().tmop_mlp_check(self._h, _s()), "tmop_mlp_check")


def features(m: mg.Mesh, x, ldf: int, first: int = 0, count: int | None = None, ldx: int | None = None, out=None):
    """bf16 patch features (as int16 tensor) of elements first..first+count-1."""
    import torch
    count = m.nelem if count is None else count
    out = torch.zeros((count, ldf), dtype=torch.int16, device=x.device) if out is None else out
    _check(lib().tmop_patch_features(m.order, m.nx[0], m.nx[1], _p(x), ldx or m.nnode, first, count, _p(out), ldf,
                                     _s()), "tmop_patch_features")
    return out


def targets(m: mg.Mesh, x0, x1, first=0, count=None, ldx=None, out=None):
    import torch
    count = m.nelem if count is None else count
    nt = n_targets(m.order)
    out = torch.zeros((count, nt), dtype=torch.float32, device=x0.device) if out is None else out
    _check(lib().tmop_patch_targets(m.order, m.nx[0], m.nx[1], _p(x0), _p(x1), ldx or m.nnode, first, count, _p(out),
                                    out.shape[1], _s()), "tmop_patch_targets")
    return out


def apply(m: mg.Mesh, x0, fixed_dev, Y, out=None, scale: float = 1.0):
    import torch
    out = torch.empty_like(x0) if out is None else out
    _check(lib().tmop_patch_apply(m.order, m.nx[0], m.nx[1], _p(x0), None if fixed_dev is None else _p(fixed_dev),
                                  m.nnode, _p(Y), Y.shape[1], float(scale), _p(out), _s()), "tmop_patch_apply")
    return out


def lattice_vertices(m: mg.Mesh, x, ldx: int, xv, ldv: int):
    _check(lib().tmop_lattice_vertices(m.order, m.nx[0], m.nx[1], _p(x), ldx, _p(xv), ldv, _s()),
           "tmop_lattice_vertices")


def lattice_prolong_add(m: mg.Mesh, xv0, xv1, ldv: int, x_in, fixed_dev, ldx: int, x_out):
    _check(lib().tmop_lattice_prolong_add(m.order, m.nx[0], m.nx[1], _p(xv0), _p(xv1), ldv, _p(x_in),
                                          None if fixed_dev is None else _p(fixed_dev), ldx, _p(x_out), _s()),
           "tmop_lattice_prolong_add")


# coarse contexts by (grid, metric, count), one cache per host thread: a
# context's workspace serves one solve at a time
_coarse_tls = threading.local()


def coarse_context(m: mg.Mesh, count: int):
    """The order-1 TMOP problem of the element vertices of `count` meshes
    shaped like m (same metric, boundary vertices fixed), one block each."""
    key = (tuple(m.nx), m.metric, count)
    _coarse_ctx = getattr(_coarse_tls, "ctx", None)
    if _coarse_ctx is None:
        _coarse_ctx = _coarse_tls.ctx = {}
    if key not in _coarse_ctx:
        xv, en, fx = mg.structured(m.dim, 1, m.nx)
        Nv = xv.shape[1]
        # one order-1 grid, or a stack of `count` of them (nodes grid after grid)
        st = list(m.nx) + ([count] if count > 1 else [])
        ctx = tm.Context(m.dim, 1, Nv * count, None, np.concatenate([fx] * count, axis=1), 3, m.metric,
                         structured=st, precision=tm.FP64, nelem=en.shape[0] * count)
        _coarse_ctx[key] = ctx
    return _coarse_ctx[key]


def coarse_stage(m: mg.Mesh, x0, fixed_dev=None, count: int = 1, out=None, max_newton=30, rtol=1e-8):
    """x0 + P (xv* - xv0) for `count` meshes shaped like m stored back to
    back in x0 ([2][count * nnode]): the element-vertex grids of all of them
    solved by Newton as one order-1 problem, each vertex displacement
    interpolated to its mesh's free nodes. Returns (x, newton result); x is
    x0 (a copy) when the coarse Newton does not converge."""
    import torch
    N, ldx = m.nnode, x0.shape[1]
    Nv = (m.nx[0] + 1) * (m.nx[1] + 1)
    ldv = Nv * count
    xv0 = torch.empty((2, ldv), dtype=torch.float64, device=x0.device)
    for i in range(count):
        lattice_vertices(m, x0[:, i * N:], ldx, xv0[:, i * Nv:], ldv)
    ctx = coarse_context(m, count)
    xv1 = xv0.clone()
    r = ctx.newton_solve(xv1, max_newton=max_newton, rtol=rtol)
    out = torch.empty_like(x0) if out is None else out
    if r.status != tm.OK:
        out.copy_(x0)
        return out, r
    for i in range(count):
        fx = None if fixed_dev is None else fixed_dev[:, i * N:]
        lattice_prolong_add(m, xv0[:, i * Nv:], xv1[:, i * Nv:], ldv, x0[:, i * N:], fx, ldx, out[:, i * N:])
    return out, r


def union_context(meshes, precision=tm.FP32_MIXED):
    """One TMOP problem made of disjoint meshes: a structured stack when
    they are 2D grids of one size (the nodes of one grid after another; the
    two-level preconditioner applies), unstructured connectivity otherwise."""
    m0 = meshes[0]
    N, B = m0.nnode, len(meshes)
    fixed = np.concatenate([m.fixed for m in meshes], axis=1)
    x = np.concatenate([m.x for m in meshes], axis=1)
    if m0.dim == 2 and all(tuple(m.nx) == tuple(m0.nx) for m in meshes):
        ctx = tm.Context(2, m0.order, N * B, None, fixed, m0.nq, m0.metric, quad_kind=m0.quad_kind,
                         structured=[m0.nx[0], m0.nx[1], B], precision=precision, nelem=B * m0.nelem)
        ctx.stacked = True
    else:
        en = np.concatenate([m.elem_nodes + i * N for i, m in enumerate(meshes)]).astype(np.int32)
        ctx = tm.Context(m0.dim, m0.order, N * B, en, fixed, m0.nq, m0.metric, quad_kind=m0.quad_kind,
                         precision=precision)
        ctx.stacked = False
    return ctx, x


@dataclass
class Dataset:
    X: object            # int16 (bf16 bits) [S, ld]
    T: object            # float32 [S, n_targets]
    meshes: int
    newton: list = field(default_factory=list)   # per chunk (status, Newton its, Krylov its, seconds)
    seconds: float = 0.0


def make_dataset(n_meshes=2000, seed0=1000, nx=32, ldf=256, chunk=50, precision=tm.FP32_MIXED,
                 preset="c5", max_newton=60, rtol=1e-10, coarse=False, workers=4) -> Dataset:
    """Newton-converged displacement targets from n_meshes seeded meshes
    (seeds seed0, seed0+1, ...), solved chunk meshes at a time as one
    block-diagonal problem, to |g| <= rtol |g0| of the chunk (far below what
    a bf16 network resolves). The chunk trades launch overhead against the
    shared Krylov space and step length of a larger union (whose MINRES must
    resolve every block's spectrum, and whose line search every block's
    validity): 50 meshes of 32^2 took 2.4x less time than 250. The chunks'
    solves are small, latency-bound kernels, so `workers` host threads run
    chunks at once, each on its own CUDA stream and context (the library's
    graph captures are thread-local); the samples keep the chunk order.
    coarse: features and targets are taken from the coarse stage's mesh
    (coarse_stage) instead of the jittered one."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    t0 = time.perf_counter()
    device = torch.cuda.current_device()

    def solve_chunk(c0):
        torch.cuda.set_device(device)
        stream = torch.cuda.Stream()
        Xc, Tc = [], []
        with torch.cuda.stream(stream):
            ms = [mg.make_mesh(preset, seed0 + i, nx=nx) for i in range(c0, min(c0 + chunk, n_meshes))]
            ctx, xh = union_context(ms, precision)
            try:
                x0 = torch.tensor(xh, device="cuda")
                if coarse:
                    fx = torch.tensor(np.concatenate([m.fixed for m in ms], axis=1), device="cuda")
                    xc, _ = coarse_stage(ms[0], x0, fx, count=len(ms))
                    if ctx.energy(xc)[2] > 0:    # valid everywhere: the base of this chunk
                        x0 = xc
                x1 = x0.clone()
                # a stack of boundary-fixed grids takes the two-level preconditioner
                pc = 2 if ctx.stacked and all(np.array_equal(m.fixed, ms[0].fixed) for m in ms) else 0
                r = ctx.newton_solve(x1, max_newton=max_newton, rtol=rtol, precond=pc)
                if r.status != tm.OK:
                    raise RuntimeError(f"data generation: Newton failed on chunk {c0}: {tm.status_string(r.status)}")
                N = ms[0].nnode
                for i, m in enumerate(ms):
                    # component stride of the union positions is the union node count
                    xa, xb = x0[:, i * N:], x1[:, i * N:]
                    Xc.append(features(m, xa, ldf, ldx=x0.shape[1]))
                    Tc.append(targets(m, xa, xb, ldx=x0.shape[1]))
            finally:
                stream.synchronize()   # nothing of this chunk in flight when its buffers are freed
                ctx.close()
        return Xc, Tc, (r.status, r.report["iterations"], r.report["krylov_iterations"])

    starts = list(range(0, n_meshes, chunk))
    if workers > 1 and len(starts) > 1:
        with ThreadPoolExecutor(max_workers=min(workers, len(starts))) as ex:
            results = list(ex.map(solve_chunk, starts))
    else:
        results = [solve_chunk(c0) for c0 in starts]
    Xs = [x for r in results for x in r[0]]
    Ts = [t for r in results for t in r[1]]
    log = [r[2] for r in results]
    torch.cuda.synchronize()
    return Dataset(torch.cat(Xs), torch.cat(Ts), n_meshes, log, time.perf_counter() - t0)


def train(net: MLP, ds: Dataset, epochs=20, batch=4096, lr=1e-3, seed=0, log_every=0, graph=True):
    """Adam on minibatches of the dataset (reshuffled every epoch). With
    graph, each epoch captures one training step (tmop_mlp_gradients +
    tmop_mlp_adam on fixed minibatch buffers, its learning rate) in a CUDA
    graph and replays it for every minibatch."""
    import torch
    S = ds.X.shape[0]
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    loss = torch.zeros((), dtype=torch.float64, device="cuda")
    Xb = torch.empty((batch, ds.X.shape[1]), dtype=ds.X.dtype, device="cuda")
    Tb = torch.empty((batch, ds.T.shape[1]), dtype=ds.T.dtype, device="cuda")
    hist = []
    nb = S // batch
    if graph and nb > 0:   # first use outside capture: workspace allocation, kernel attributes
        torch.index_select(ds.X, 0, torch.arange(batch, device="cuda"), out=Xb)
        torch.index_select(ds.T, 0, torch.arange(batch, device="cuda"), out=Tb)
        net.gradients(Xb, Tb, loss)
        torch.cuda.synchronize()
    for ep in range(epochs):
        perm = torch.randperm(S, device="cuda", generator=g)
        acc = 0.0
        lr_ep = float(lr * 0.5 * (1 + np.cos(np.pi * ep / epochs)))      # cosine decay
        step = None
        if graph and nb > 0:
            step = torch.cuda.CUDAGraph()
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side), torch.cuda.graph(step, stream=side):
                net.gradients(Xb, Tb, loss)
                net.adam(lr_ep)
            torch.cuda.current_stream().wait_stream(side)
        for b in range(nb):
            idx = perm[b * batch:(b + 1) * batch]
            torch.index_select(ds.X, 0, idx, out=Xb)
            torch.index_select(ds.T, 0, idx, out=Tb)
            if step is not None:
                step.replay()
            else:
                net.gradients(Xb, Tb, loss)
                net.adam(lr_ep)
            if b % 50 == 0 or b == nb - 1:
                acc = loss.item()
        net.check()
        hist.append(acc)
        if log_every and ep % log_every == 0:
            print(f"epoch {ep} loss {acc:.4e}")
    return hist


@dataclass
class Proposal:
    x: object
    used: bool
    F0: float
    F: float
    min_detA: float
    scale: float = 1.0   # the damping that was kept (0: no network step)
    coarse: bool = False  # started from the coarse stage


def propose(net: MLP, m: mg.Mesh, ctx: tm.Context, x0, fixed_dev, scales=(1.0, 0.5, 0.25),
            coarse=False) -> Proposal:
    """Proposal with fallback: the first of b + s h Y (s in scales) with
    min det A > 0 and F below F(x0) is kept, where b is x0 or, with coarse,
    the coarse stage's mesh (then b alone is the last candidate); otherwise
    Newton starts from x0."""
    import torch
    S = m.nelem
    Sp = (S + 63) // 64 * 64
    _, F0, _ = ctx.energy(x0)
    base = x0
    if coarse:
        xc, rc_ = coarse_stage(m, x0, fixed_dev)
        if rc_.status == tm.OK:
            base = xc
    X = torch.zeros((Sp, net.ld), dtype=torch.int16, device=x0.device)
    features(m, base, net.ld, out=X[:S])
    Y = net.forward(X)[:S].contiguous()
    F, md = float("inf"), 0.0
    for sc in scales:
        xp = apply(m, base, fixed_dev, Y, scale=sc)
        rc, F, md = ctx.energy(xp)
        if rc == tm.OK and md > 0 and F < F0:
            return Proposal(xp, True, F0, F, md, sc, coarse=base is not x0)
    if base is not x0:
        rc, F, md = ctx.energy(base)
        if rc == tm.OK and md > 0 and F < F0:
            return Proposal(base.clone(), True, F0, F, md, 0.0, coarse=True)
    return Proposal(x0, False, F0, F, md, 0.0)
