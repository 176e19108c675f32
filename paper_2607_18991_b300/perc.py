"""Python binding of libperc.so (include/perc.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; PyTorch provides device memory
and the stream.  The names follow the C entry points: ``rank``, ``nstar``, ``mass``, ``check``,
``mlp_forward``, ``mlp_grad``, ``adam``, ``mlp_train``, ``bracket``.  If the shared library is
missing this module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libperc.so")
NEVER = 0xFFFFFFFF
MAX_L = 73
OP_RANK, OP_NSTAR, OP_MASS, OP_SMAX, OP_PERIODIC, OP_NSTAR_ANY, OP_MINIMAX = 1, 2, 3, 4, 5, 6, 7
PERIODIC_MAX_L = 40
AXIS_SHIFT, NUM_AXES = 8, 5  # zone word: spanning axis in bits 8..10; axes x1..x5
OPT_THREADS, OPT_SMEM_NODES, OPT_MAX_CTAS, OPT_GROUP, OPT_METHOD, OPT_SPIN_LIMIT = 1, 2, 3, 4, 5, 6
METHOD_AUTO, METHOD_BISECTION, METHOD_SWEEP = 0, 1, 2
MLP_NPARAM = 4931
MB_L2_READ, MB_SMEM_READ, MB_SMEM_ATOMIC, MB_SMEM_CAS, MB_L2_ATOMIC = 1, 2, 3, 4, 5
STATS_FIELDS = ("passes", "new_sites", "probe_sites", "hooks", "early_exits", "fallbacks",
                "verified", "sites_merged", "unions", "cyc_setup", "cyc_update", "cyc_union",
                "cyc_commit", "cyc_scan", "cyc_link", "chunks")

_lib = None


class PercError(RuntimeError):
    def __init__(self, rc: int, what: str):
        super().__init__(f"{what}: {status_string(rc)} ({rc})")
        self.rc = rc


def lib() -> ctypes.CDLL:
    """Load libperc.so (built by ``paper_2607_18991_b300.build``); raise if it is not there."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libperc.so not built ({LIB_PATH}); run paper_2607_18991_b300/build.py")
    L = ctypes.CDLL(LIB_PATH)
    vp, u32, u64, i32, sz, f32 = (ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int,
                                  ctypes.c_size_t, ctypes.c_float)
    sig = {
        "perc_workspace_bytes": (sz, [i32, u32, u32]),
        "perc_rank": (i32, [u32, vp, u32, vp, vp, vp, sz, vp]),
        "perc_nstar": (i32, [vp, u32, u32, vp, vp, vp, vp, vp, sz, vp]),
        "perc_nstar_noalloc": (i32, [vp, u32, u32, vp, vp, vp, vp, vp]),
        "perc_nstar_any": (i32, [vp, u32, u32, vp, vp, vp, vp, vp, sz, vp]),
        "perc_nstar_min_axes": (i32, [vp, u32, u32, vp, vp]),
        "perc_mass_periodic": (i32, [vp, u32, u32, vp, vp, vp, sz, vp]),
        "perc_nstar_wrap": (i32, [vp, u32, u32, vp, vp, sz, vp]),
        "perc_mass": (i32, [vp, u32, u32, vp, vp, vp, sz, vp]),
        "perc_smax_window": (i32, [vp, u32, u32, vp, vp, u32, vp, vp, sz, vp]),
        "perc_binomial_weights": (i32, [vp, vp, vp, u32, u32, vp, u32, vp, vp]),
        "perc_pmax": (i32, [vp, vp, u32, u32, vp, vp, vp, u32, u32, vp, vp]),
        "perc_check": (i32, [vp, vp]),
        "perc_set_launch_option": (i32, [i32, i32]),
        "perc_mlp_forward": (i32, [vp, vp, u32, vp, vp]),
        "perc_mlp_grad": (i32, [vp, vp, vp, u32, vp, vp, vp]),
        "perc_adam": (i32, [vp, vp, vp, vp, u32, u32, f32, f32, f32, f32, vp]),
        "perc_mlp_train": (i32, [vp, vp, vp, vp, vp, vp, u32, u32, u32, f32, vp, vp]),
        "perc_bracket": (i32, [vp, vp, u32, f32, vp, vp]),
        "perc_status_string": (ctypes.c_char_p, [i32]),
        "perc_microbench": (i32, [i32, vp, sz, u32, ctypes.POINTER(ctypes.c_double), vp]),
        "perc_prefix_share": (i32, [vp, u32, vp, vp, vp]),
        "perc_rank_prefix": (i32, [u32, vp, u32, vp, vp, vp, vp, sz, vp]),
        "perc_nstar_prefix": (i32, [vp, u32, u32, vp, vp, vp, vp, vp, vp, vp, sz, vp]),
        "perc_nstar_any_prefix": (i32, [vp, u32, u32, vp, vp, vp, vp, vp, vp, vp, sz, vp]),
        "perc_prefix_shares": (i32, [vp, u32, vp, vp, u32, u32, vp, vp]),
        "perc_rank_prefix_seeds": (i32, [u32, vp, u32, vp, vp, vp, vp, sz, vp]),
        "perc_nstar_minimax": (i32, [vp, u32, u32, vp, vp, sz, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def exported_symbols() -> list[str]:
    return ["perc_workspace_bytes", "perc_rank", "perc_nstar", "perc_nstar_any", "perc_nstar_noalloc",
            "perc_nstar_min_axes", "perc_mass",
            "perc_mass_periodic", "perc_nstar_wrap", "perc_microbench",
            "perc_smax_window", "perc_binomial_weights", "perc_pmax", "perc_check",
            "perc_mlp_forward", "perc_mlp_grad", "perc_adam", "perc_mlp_train", "perc_bracket",
            "perc_status_string", "perc_set_launch_option", "perc_prefix_share", "perc_rank_prefix",
            "perc_nstar_prefix", "perc_nstar_any_prefix", "perc_prefix_shares", "perc_rank_prefix_seeds",
            "perc_nstar_minimax"]


def status_string(rc: int) -> str:
    return lib().perc_status_string(rc).decode()


def _ok(rc: int, what: str):
    if rc != 0:
        raise PercError(rc, what)


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def set_launch_option(option: int, value: int):
    _ok(lib().perc_set_launch_option(option, value), "perc_set_launch_option")


def workspace_bytes(op: int, max_L: int, num: int) -> int:
    return int(lib().perc_workspace_bytes(op, max_L, num))


def new_workspace(nbytes: int, device="cuda") -> torch.Tensor:
    """A workspace buffer of nbytes with its 256-byte header (status word, work queue) zeroed."""
    buf = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
    buf[:256].zero_()
    return buf


class Workspace:
    """Caller-owned scratch for the library, grown on demand (a torch uint8 tensor)."""

    def __init__(self, device="cuda"):
        self.device = torch.device(device)
        self.buf = None

    def get(self, nbytes: int) -> torch.Tensor:
        if nbytes <= 0:
            raise PercError(-1, "workspace size query")
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = None
            self.buf = new_workspace(nbytes, self.device)
        return self.buf


_default_ws: dict = {}


def default_workspace(device=None) -> Workspace:
    dev = torch.device(device if device is not None else "cuda")
    key = (dev.type, dev.index if dev.index is not None else torch.cuda.current_device())
    if key not in _default_ws:
        _default_ws[key] = Workspace(dev)
    return _default_ws[key]


# ------------------------------------------------------------------------------------------------
# perc_rank / samples
# ------------------------------------------------------------------------------------------------
def rank(L: int, seeds, ws: Workspace | None = None, stream=None, out=None):
    """(perm, rank), int32 tensors [len(seeds), L^5] on the GPU (values are uint32 < 2^31)."""
    seeds_t = torch.as_tensor(np.asarray(seeds, dtype=np.uint64).astype(np.int64), device="cuda")
    S = seeds_t.numel()
    N = L ** 5
    if out is None:
        perm = torch.empty((S, N), dtype=torch.int32, device="cuda")
        rk = torch.empty((S, N), dtype=torch.int32, device="cuda")
    else:
        perm, rk = out
    ws = ws or default_workspace()
    nb = workspace_bytes(OP_RANK, L, S)
    buf = ws.get(nb)
    _ok(lib().perc_rank(L, seeds_t.data_ptr(), S, perm.data_ptr(), rk.data_ptr(), buf.data_ptr(),
                        buf.numel(), _stream(stream)), "perc_rank")
    return perm, rk


def zone_word(masks, axes=0):
    """perc_sample.zone_mask: zone bits 0..6 and the spanning axis (0..4) in bits 8..10."""
    return np.asarray(masks, dtype=np.int64) | (np.asarray(axes, dtype=np.int64) << AXIS_SHIFT)


def make_samples(Ls, masks, perm_ptrs, rank_ptrs) -> torch.Tensor:
    """Device array of perc_sample {uint32 L, uint32 zone word, perm*, rank*} as int64 [num, 3];
    `masks` are zone words (a plain zone mask 1..127 spans along x1)."""
    Ls = np.asarray(Ls, dtype=np.int64)
    masks = np.asarray(masks, dtype=np.int64)
    arr = np.zeros((len(Ls), 3), dtype=np.int64)
    arr[:, 0] = Ls | (masks << 32)
    arr[:, 1] = np.asarray(perm_ptrs, dtype=np.uint64).astype(np.int64)
    arr[:, 2] = np.asarray(rank_ptrs, dtype=np.uint64).astype(np.int64)
    return torch.from_numpy(arr).to("cuda")


def samples_for(L: int, masks, seed_rows, perm: torch.Tensor, rk: torch.Tensor) -> torch.Tensor:
    """Samples (L, masks[k]) whose order is row seed_rows[k] of (perm, rank)."""
    N = L ** 5
    seed_rows = np.asarray(seed_rows, dtype=np.int64)
    pp = perm.data_ptr() + seed_rows * N * 4
    rp = rk.data_ptr() + seed_rows * N * 4
    return make_samples(np.full(len(seed_rows), L), masks, pp, rp)


def u32(t: torch.Tensor) -> np.ndarray:
    """int32 tensor holding uint32 values -> numpy uint32."""
    return t.cpu().numpy().view(np.uint32)


# ------------------------------------------------------------------------------------------------
# perc_nstar / perc_mass / perc_check
# ------------------------------------------------------------------------------------------------
def nstar(samples: torch.Tensor, max_L: int, bracket: torch.Tensor | None = None,
          stats: torch.Tensor | None = None, ws: Workspace | None = None, stream=None,
          out=None, want_passes: bool = True):
    """(nstar, passes): int32 tensors [num] (uint32 values; PERC_NEVER = -1 as int32)."""
    num = samples.shape[0]
    if out is None:
        ns = torch.empty(num, dtype=torch.int32, device="cuda")
        ps = torch.empty(num, dtype=torch.int32, device="cuda") if want_passes else None
    else:
        ns, ps = out
    ws = ws or default_workspace()
    buf = ws.get(workspace_bytes(OP_NSTAR, max_L, num))
    _ok(lib().perc_nstar(samples.data_ptr(), num, max_L, _ptr(bracket), ns.data_ptr(), _ptr(ps),
                         _ptr(stats), buf.data_ptr(), buf.numel(), _stream(stream)), "perc_nstar")
    return ns, ps


def nstar_any(samples: torch.Tensor, max_L: int, bracket: torch.Tensor | None = None,
              stats: torch.Tensor | None = None, ws: Workspace | None = None, stream=None, out=None,
              want_passes: bool = True):
    """perc_nstar_any: n* for spanning along any axis, one sweep per sample; (nstar, passes)."""
    num = samples.shape[0]
    if out is None:
        ns = torch.empty(num, dtype=torch.int32, device="cuda")
        ps = torch.empty(num, dtype=torch.int32, device="cuda") if want_passes else None
    else:
        ns, ps = out
    ws = ws or default_workspace()
    buf = ws.get(workspace_bytes(OP_NSTAR_ANY, max_L, num))
    _ok(lib().perc_nstar_any(samples.data_ptr(), num, max_L, _ptr(bracket), ns.data_ptr(), _ptr(ps), _ptr(stats),
                             buf.data_ptr(), buf.numel(), _stream(stream)), "perc_nstar_any")
    return ns, ps


def nstar_min_axes(nstar_axes: torch.Tensor, axes: int = NUM_AXES, out=None, stream=None) -> torch.Tensor:
    """perc_nstar_min_axes: n* for spanning along any axis from per-axis n* stored [num][axes]
    (int32 tensors holding uint32; PERC_NEVER = -1)."""
    num = nstar_axes.numel() // axes
    o = out if out is not None else torch.empty(num, dtype=torch.int32, device="cuda")
    _ok(lib().perc_nstar_min_axes(nstar_axes.data_ptr(), num, axes, o.data_ptr(), _stream(stream)),
        "perc_nstar_min_axes")
    return o


def mass_periodic(samples: torch.Tensor, max_L: int, n: torch.Tensor, ws: Workspace | None = None,
                  stream=None, out=None):
    """perc_mass_periodic: S_max(n) on the torus (offsets wrap modulo L), int64 tensor [num]."""
    num = samples.shape[0]
    m = out if out is not None else torch.empty(num, dtype=torch.int64, device="cuda")
    n = n.to(device="cuda", dtype=torch.int64).contiguous()
    ws = ws or default_workspace()
    buf = ws.get(workspace_bytes(OP_PERIODIC, max_L, num))
    _ok(lib().perc_mass_periodic(samples.data_ptr(), num, max_L, n.data_ptr(), m.data_ptr(), buf.data_ptr(),
                                 buf.numel(), _stream(stream)), "perc_mass_periodic")
    return m


def nstar_wrap(samples: torch.Tensor, max_L: int, ws: Workspace | None = None, stream=None, out=None):
    """perc_nstar_wrap: first n at which a cluster wraps around the torus along each sample's axis,
    int32 tensor [num] of uint32 values."""
    num = samples.shape[0]
    ns = out if out is not None else torch.empty(num, dtype=torch.int32, device="cuda")
    ws = ws or default_workspace()
    buf = ws.get(workspace_bytes(OP_PERIODIC, max_L, num))
    _ok(lib().perc_nstar_wrap(samples.data_ptr(), num, max_L, ns.data_ptr(), buf.data_ptr(), buf.numel(),
                              _stream(stream)), "perc_nstar_wrap")
    return ns


def nstar_noalloc(samples: torch.Tensor, max_L: int, bracket: torch.Tensor | None = None,
                  stats: torch.Tensor | None = None, stream=None):
    """perc_nstar_noalloc: n* and passes with the library's own static scratch (no workspace)."""
    num = samples.shape[0]
    ns = torch.empty(num, dtype=torch.int32, device="cuda")
    ps = torch.empty(num, dtype=torch.int32, device="cuda")
    _ok(lib().perc_nstar_noalloc(samples.data_ptr(), num, max_L, _ptr(bracket), ns.data_ptr(), ps.data_ptr(),
                                 _ptr(stats), _stream(stream)), "perc_nstar_noalloc")
    return ns, ps


def mass(samples: torch.Tensor, max_L: int, n: torch.Tensor, ws: Workspace | None = None,
         stream=None, out=None):
    """S_max(n) per sample, int64 tensor [num]."""
    num = samples.shape[0]
    m = out if out is not None else torch.empty(num, dtype=torch.int64, device="cuda")
    ws = ws or default_workspace()
    buf = ws.get(workspace_bytes(OP_MASS, max_L, num))
    n = n.to(device="cuda", dtype=torch.int64).contiguous()
    _ok(lib().perc_mass(samples.data_ptr(), num, max_L, n.data_ptr(), m.data_ptr(), buf.data_ptr(),
                        buf.numel(), _stream(stream)), "perc_mass")
    return m


def smax_window(samples: torch.Tensor, max_L: int, n_lo: torch.Tensor, window: int,
                count: torch.Tensor | None = None, ws: Workspace | None = None, stream=None,
                out=None) -> torch.Tensor:
    """S_max(n_lo[k] + j), j < count[k] (all `window` entries when count is None), per sample:
    int32 tensor [num, window] of uint32 values (0 past count[k] or past L^5)."""
    num = samples.shape[0]
    sm = out if out is not None else torch.empty((num, window), dtype=torch.int32, device="cuda")
    ws = ws or default_workspace()
    buf = ws.get(workspace_bytes(OP_SMAX, max_L, num))
    n_lo = n_lo.to(device="cuda", dtype=torch.int64).contiguous()
    if count is not None:
        count = count.to(device="cuda", dtype=torch.int32).contiguous()
    _ok(lib().perc_smax_window(samples.data_ptr(), num, max_L, n_lo.data_ptr(), _ptr(count), window,
                               sm.data_ptr(), buf.data_ptr(), buf.numel(), _stream(stream)), "perc_smax_window")
    return sm


def binomial_weights(N: torch.Tensor, n_lo: torch.Tensor, window: int, p: torch.Tensor,
                     count: torch.Tensor | None = None, stream=None, out=None) -> torch.Tensor:
    """B(N[g], n_lo[g] + k, p[g, j]) for k < count[g] (all k < window when count is None), as
    float64 [groups, np, window] (0 elsewhere)."""
    N = N.to(device="cuda", dtype=torch.int64).contiguous()
    n_lo = n_lo.to(device="cuda", dtype=torch.int64).contiguous()
    p = p.to(device="cuda", dtype=torch.float64).contiguous()
    if count is not None:
        count = count.to(device="cuda", dtype=torch.int32).contiguous()
    G, npr = p.shape
    w = out if out is not None else torch.empty((G, npr, window), dtype=torch.float64, device="cuda")
    _ok(lib().perc_binomial_weights(N.data_ptr(), n_lo.data_ptr(), _ptr(count), G, window, p.data_ptr(), npr,
                                    w.data_ptr(), _stream(stream)), "perc_binomial_weights")
    return w


def pmax(smax: torch.Tensor, group: torch.Tensor, w: torch.Tensor, N: torch.Tensor,
         count: torch.Tensor | None = None, stream=None, out=None) -> torch.Tensor:
    """P_max(p) per (sample, p): float64 [num, np] from S_max windows and weight groups."""
    num, window = smax.shape
    G, npr, W = w.shape
    assert W == window
    group = group.to(device="cuda", dtype=torch.int32).contiguous()
    N = N.to(device="cuda", dtype=torch.int64).contiguous()
    if count is not None:
        count = count.to(device="cuda", dtype=torch.int32).contiguous()
    pm = out if out is not None else torch.empty((num, npr), dtype=torch.float64, device="cuda")
    _ok(lib().perc_pmax(smax.data_ptr(), group.data_ptr(), num, window, w.data_ptr(), N.data_ptr(), _ptr(count),
                        G, npr, pm.data_ptr(), _stream(stream)), "perc_pmax")
    return pm


def check(ws: Workspace | None = None, stream=None) -> int:
    ws = ws or default_workspace()
    if ws.buf is None:
        return 0
    return int(lib().perc_check(ws.buf.data_ptr(), _stream(stream)))


def new_stats() -> torch.Tensor:
    return torch.zeros(len(STATS_FIELDS), dtype=torch.int64, device="cuda")


def stats_dict(stats: torch.Tensor) -> dict:
    return dict(zip(STATS_FIELDS, (int(x) for x in stats.cpu().tolist())))


# ------------------------------------------------------------------------------------------------
# bracket network
# ------------------------------------------------------------------------------------------------
def mlp_forward(params: torch.Tensor, X: torch.Tensor, stream=None) -> torch.Tensor:
    B = X.shape[0]
    Q = torch.empty((B, 3), dtype=torch.float32, device="cuda")
    _ok(lib().perc_mlp_forward(params.data_ptr(), X.data_ptr(), B, Q.data_ptr(), _stream(stream)),
        "perc_mlp_forward")
    return Q


def mlp_grad(params: torch.Tensor, X: torch.Tensor, y: torch.Tensor, stream=None):
    grad = torch.empty(MLP_NPARAM, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    _ok(lib().perc_mlp_grad(params.data_ptr(), X.data_ptr(), y.data_ptr(), X.shape[0], grad.data_ptr(),
                            loss.data_ptr(), _stream(stream)), "perc_mlp_grad")
    return grad, loss


def adam(params, grad, m, v, t: int, lr: float, b1=0.9, b2=0.999, eps=1e-8, stream=None):
    _ok(lib().perc_adam(params.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), params.numel(),
                        t, lr, b1, b2, eps, _stream(stream)), "perc_adam")


def mlp_train(params, m, v, X, y, t0: int, steps: int, lr: float, stream=None) -> torch.Tensor:
    grad = torch.empty(MLP_NPARAM, dtype=torch.float32, device="cuda")
    losses = torch.empty(max(steps, 1), dtype=torch.float32, device="cuda")
    _ok(lib().perc_mlp_train(params.data_ptr(), m.data_ptr(), v.data_ptr(), grad.data_ptr(), X.data_ptr(),
                             y.data_ptr(), X.shape[0], t0, steps, lr, losses.data_ptr(), _stream(stream)),
        "perc_mlp_train")
    return losses[:steps]


def bracket(params: torch.Tensor, samples: torch.Tensor, margin: float = 0.0, stream=None,
            out=None) -> torch.Tensor:
    num = samples.shape[0]
    br = out if out is not None else torch.empty((num, 2), dtype=torch.int32, device="cuda")
    _ok(lib().perc_bracket(params.data_ptr(), samples.data_ptr(), num, margin, br.data_ptr(),
                           _stream(stream)), "perc_bracket")
    return br


def microbench(which: int, buf: torch.Tensor, iters: int, stream=None) -> float:
    """perc_microbench: enqueue one on-chip throughput probe over buf; returns its units (bytes or
    operations) -- the caller times the launch."""
    units = ctypes.c_double()
    _ok(lib().perc_microbench(which, buf.data_ptr(), buf.numel() * buf.element_size(), iters, ctypes.byref(units),
                              _stream(stream)), "perc_microbench")
    return units.value


def prefix_sites(N: int, share: int) -> int:
    """PERC_PREFIX_SITES: sites of an order that perc_rank_prefix ranks at least for `share`."""
    base = (int(N) * min(int(share), 1 << 24)) >> 24
    return min(int(N), base * 9 // 8 + 64)


def nstar_minimax(samples: torch.Tensor, max_L: int, ws: Workspace | None = None, stream=None) -> torch.Tensor:
    """perc_nstar_minimax: n* as a min-max path value (int32 tensor [num], uint32 values)."""
    num = samples.shape[0]
    out = torch.empty(num, dtype=torch.int32, device=samples.device)
    ws = ws or default_workspace()
    buf = ws.get(workspace_bytes(OP_MINIMAX, max_L, num))
    _ok(lib().perc_nstar_minimax(samples.data_ptr(), num, max_L, out.data_ptr(), buf.data_ptr(), buf.numel(),
                                 _stream(stream)), "perc_nstar_minimax")
    return out
