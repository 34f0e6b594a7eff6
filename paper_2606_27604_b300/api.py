"""Python binding of libsss (include/sss.h): argument marshalling only.

Every step of the walk runs in the library's CUDA kernels; this module only
turns torch CUDA tensors into the C structs and pointers the C ABI takes.
Importing it loads ``libsss.so`` and raises if the library is missing --
there is no CPU fallback.
"""
import ctypes as C
import os
from dataclasses import dataclass, asdict
from typing import Optional

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsss.so")

SSS_OK = 0
STATUS_NAMES = {0: "SSS_OK", 1: "SSS_ERR_INVALID_ARG", 2: "SSS_ERR_CUDA",
                3: "SSS_ERR_WORKSPACE", 4: "SSS_ERR_STEP_LIMIT", 5: "SSS_ERR_OVERFLOW",
                6: "SSS_ERR_DEVICE_PARAM", 7: "SSS_ERR_UNSUPPORTED", 8: "SSS_ERR_TIMEOUT",
                9: "SSS_ERR_TOO_LARGE"}
FLAG_PARAM, FLAG_STEP_LIMIT, FLAG_OVERFLOW, FLAG_ZERO_WEIGHT = 0x1, 0x2, 0x4, 0x8


class SSSError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {STATUS_NAMES.get(code, code)} ({_status_string(code)})")


class Params(C.Structure):
    _fields_ = [("alpha", C.c_void_p), ("sigma_t", C.c_void_p), ("g", C.c_void_p),
                ("w", C.c_void_p), ("n_paths", C.c_void_p), ("uniform_paths", C.c_uint32),
                ("thickness_mm", C.c_void_p), ("n_rel", C.c_float), ("K", C.c_int32),
                ("n_inst", C.c_int64), ("alpha2", C.c_void_p), ("sigma_t2", C.c_void_p),
                ("g2", C.c_void_p), ("d1_mm", C.c_void_p)]


class Opts(C.Structure):
    _fields_ = [("nbins", C.c_int32), ("r_max_mm", C.c_float), ("mode", C.c_int32),
                ("rr_threshold", C.c_float), ("entry_fresnel", C.c_int32),
                ("max_steps", C.c_uint32), ("seed", C.c_uint64), ("path_offset", C.c_uint32),
                ("want_sumsq", C.c_int32), ("schedule", C.c_int32), ("use_graph", C.c_int32),
                ("block_threads", C.c_int32), ("unit_paths", C.c_int32),
                ("regroup", C.c_int32), ("instance_offset", C.c_uint32),
                ("incidence", C.c_int32), ("log_r_min_mm", C.c_float),
                ("select_pdf", C.c_int32), ("hero_bands", C.c_int32),
                ("hero_texel_bands", C.c_int32), ("hero_orbits", C.c_int32)]


TALLY_KEYS = ("R", "T", "A", "bins", "overflow", "R_k", "R1", "stderr_R", "stderr_bins",
              "truncated", "steps", "raw", "profile")


class Tallies(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in TALLY_KEYS]


class GradIn(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("grad_R", "grad_bins", "grad_R_k", "grad_T")]


GRAD_KEYS = ("d_alpha", "d_sigma_t", "d_g", "d_w", "d_alpha2", "d_sigma_t2", "d_g2")


class GradOut(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in GRAD_KEYS]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libsss.so not built at {LIB_PATH}; run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    lib.sss_walk_opts_default.argtypes = [C.POINTER(Opts)]
    lib.sss_walk_opts_default.restype = None
    lib.sss_tally_count.argtypes = [C.c_int32, C.c_int32, C.c_int32]
    lib.sss_tally_count.restype = C.c_int32
    for f in ("sss_walk_workspace_size", "sss_walk_bwd_workspace_size"):
        getattr(lib, f).argtypes = [C.POINTER(Params), C.POINTER(Opts)]
        getattr(lib, f).restype = C.c_size_t
    lib.sss_walk.argtypes = [C.POINTER(Params), C.POINTER(Opts), C.c_void_p, C.c_size_t,
                             C.POINTER(Tallies), C.c_void_p]
    lib.sss_walk.restype = C.c_int
    lib.sss_walk_bwd.argtypes = [C.POINTER(Params), C.POINTER(Opts), C.c_void_p, C.c_size_t,
                                 C.POINTER(GradIn), C.POINTER(GradOut), C.c_void_p]
    lib.sss_walk_bwd.restype = C.c_int
    lib.sss_read_status.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(C.c_uint32)]
    lib.sss_read_status.restype = C.c_int
    lib.sss_philox.argtypes = [C.c_void_p, C.c_uint64, C.c_int64, C.c_void_p, C.c_void_p]
    lib.sss_philox.restype = C.c_int
    lib.sss_profile_events.argtypes = [C.c_void_p, C.c_void_p]
    lib.sss_profile_events.restype = None
    lib.sss_release_plans.argtypes = []
    lib.sss_release_plans.restype = None
    lib.sss_status_string.argtypes = [C.c_int]
    lib.sss_status_string.restype = C.c_char_p
    lib.sss_probe.argtypes = [C.c_int32, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p]
    lib.sss_probe.restype = C.c_int
    lib.sss_probe_ops_per_thread_iter.argtypes = [C.c_int32]
    lib.sss_probe_ops_per_thread_iter.restype = C.c_int64
    lib.sss_last_device_status.argtypes = [C.c_void_p, C.POINTER(C.c_uint32)]
    lib.sss_last_device_status.restype = C.c_int
    lib.sss_selftest_bounded_wait.argtypes = [C.c_void_p, C.c_int64, C.c_void_p]
    lib.sss_selftest_bounded_wait.restype = C.c_int
    lib.sss_abi_version.argtypes = []
    lib.sss_abi_version.restype = C.c_int32
    if lib.sss_abi_version() != ABI_VERSION:
        raise ImportError(f"{LIB_PATH}: ABI version {lib.sss_abi_version()}, binding expects "
                          f"{ABI_VERSION}; rebuild the library")
    return lib


ABI_VERSION = 3  # struct layouts below match this version of the C header

lib = _load()


def _status_string(code: int) -> str:
    return lib.sss_status_string(code).decode()


def _check(code: int, what: str):
    if code != SSS_OK:
        raise SSSError(code, what)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


@dataclass
class WalkOptions:
    """Mirror of sss_walk_opts; see include/sss.h for the meaning of each."""
    nbins: int = 64
    r_max_mm: float = 10.0
    mode: int = 0
    rr_threshold: float = 1.0 / 16.0
    entry_fresnel: int = 1
    max_steps: int = 1 << 16
    seed: int = 0
    path_offset: int = 0
    want_sumsq: int = 1
    schedule: int = 0
    use_graph: int = 0
    block_threads: int = 0
    unit_paths: int = 0
    regroup: int = 0
    instance_offset: int = 0
    incidence: int = 0
    log_r_min_mm: float = 0.0
    select_pdf: int = 0
    hero_bands: int = 0
    hero_texel_bands: int = 0
    hero_orbits: int = 0

    def c(self) -> Opts:
        return Opts(**asdict(self))


@dataclass
class Media:
    """Device-side walk inputs (torch CUDA tensors), layouts as in sss_params."""
    alpha: torch.Tensor         # float32 [K][n]
    sigma_t: torch.Tensor
    g: torch.Tensor
    w: torch.Tensor
    n_paths: Optional[torch.Tensor] = None    # int32 (as uint32) [n] or None
    uniform_paths: int = 0
    thickness_mm: Optional[torch.Tensor] = None
    n_rel: float = 1.0
    # optional second layer of a two-layer slab: float32 [n] each
    layer2: Optional[tuple] = None   # (alpha2, sigma_t2, g2, d1_mm)

    @property
    def K(self) -> int:
        return int(self.alpha.shape[0])

    @property
    def n_inst(self) -> int:
        return int(self.alpha.shape[1])

    def c(self) -> Params:
        for t in (self.alpha, self.sigma_t, self.g, self.w):
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
                    and tuple(t.shape) == (self.K, self.n_inst)):
                raise ValueError("media arrays must be contiguous float32 CUDA [K][n_inst]")
        if self.n_paths is not None:
            assert self.n_paths.is_cuda and self.n_paths.dtype == torch.int32
            assert self.n_paths.numel() == self.n_inst
        if self.thickness_mm is not None:
            assert self.thickness_mm.is_cuda and self.thickness_mm.dtype == torch.float32
        l2 = self.layer2 if self.layer2 is not None else (None,) * 4
        for t in l2:
            if t is not None:
                assert t.is_cuda and t.dtype == torch.float32 and t.numel() == self.n_inst
        return Params(_ptr(self.alpha), _ptr(self.sigma_t), _ptr(self.g), _ptr(self.w),
                      _ptr(self.n_paths), self.uniform_paths, _ptr(self.thickness_mm),
                      self.n_rel, self.K, self.n_inst, *(_ptr(t) for t in l2))

    @staticmethod
    def from_inputs(x, device="cuda", per_instance_paths: bool = None) -> "Media":
        """From a ``paper_2606_27604_b300.inputs.WalkInputs`` (host numpy)."""
        import numpy as np
        dev = torch.device(device)
        f = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(dev)
        if per_instance_paths is None:
            uniform = x.n_paths.size > 0 and bool(np.all(x.n_paths == x.n_paths[0]))
        else:
            uniform = not per_instance_paths
        n_paths = None if uniform else torch.from_numpy(
            np.ascontiguousarray(x.n_paths, np.uint32).view(np.int32)).to(dev)
        l2 = getattr(x, "layer2", None)
        return Media(f(x.alpha), f(x.sigma_t), f(x.g), f(x.w), n_paths,
                     int(x.n_paths[0]) if uniform else 0,
                     None if x.thickness_mm is None else f(x.thickness_mm), float(x.n_rel),
                     None if l2 is None else tuple(f(a) for a in l2))


def tally_count(nbins: int, K: int, want_sumsq: int) -> int:
    return lib.sss_tally_count(nbins, K, want_sumsq)


def workspace_bytes(m: Media, o: WalkOptions, adjoint: bool = False) -> int:
    p, oc = m.c(), o.c()
    f = lib.sss_walk_bwd_workspace_size if adjoint else lib.sss_walk_workspace_size
    n = f(C.byref(p), C.byref(oc))
    if n == 0:
        raise SSSError(1, "workspace size")
    return n


def alloc_workspace(m: Media, o: WalkOptions, adjoint: bool = False) -> torch.Tensor:
    n = workspace_bytes(m, o, adjoint)
    return torch.empty(n, dtype=torch.uint8, device=m.alpha.device)


def alloc_tallies(m: Media, o: WalkOptions, raw: bool = False) -> dict:
    n, K, nb = m.n_inst, m.K, o.nbins
    dev = m.alpha.device
    d = lambda *s: torch.empty(*s, dtype=torch.float64, device=dev)
    out = {"R": d(n), "T": d(n), "A": d(n), "bins": d(n, nb), "overflow": d(n),
           "R_k": d(n, K), "R1": d(n), "steps": d(n),
           "truncated": torch.empty(n, dtype=torch.int64, device=dev)}
    if o.want_sumsq:
        out["stderr_R"] = d(n)
        out["stderr_bins"] = d(n, nb)
    if raw:
        out["raw"] = torch.empty(n, tally_count(nb, K, o.want_sumsq), dtype=torch.int64,
                                 device=dev)
    return out


def walk(m: Media, o: WalkOptions, workspace: Optional[torch.Tensor] = None,
         out: Optional[dict] = None, raw: bool = False, stream=None) -> dict:
    """Forward tallies (sss_walk).  Returns dict of CUDA tensors."""
    if workspace is None:
        workspace = alloc_workspace(m, o)
    if out is None:
        out = alloc_tallies(m, o, raw)
    t = Tallies(**{k: _ptr(out.get(k)) for k in TALLY_KEYS})
    p, oc = m.c(), o.c()
    _check(lib.sss_walk(C.byref(p), C.byref(oc), _ptr(workspace), workspace.numel(),
                        C.byref(t), _stream(stream)), "sss_walk")
    out["_workspace"] = workspace
    return out


def walk_bwd(m: Media, o: WalkOptions, grad_R=None, grad_bins=None, grad_R_k=None,
             grad_T=None, workspace: Optional[torch.Tensor] = None, out: Optional[dict] = None,
             stream=None) -> dict:
    """Path-replay adjoint (sss_walk_bwd): d(sum upstream * tallies)/d(media).
    With a second layer the result also holds d_alpha2, d_sigma_t2, d_g2
    ([n_inst]) for the layer's optics."""
    if workspace is None:
        workspace = alloc_workspace(m, o, adjoint=True)
    dev = m.alpha.device
    if out is None:
        out = {k: torch.empty(m.K, m.n_inst, dtype=torch.float64, device=dev)
               for k in ("d_alpha", "d_sigma_t", "d_g", "d_w")}
        if m.layer2 is not None:
            for k in ("d_alpha2", "d_sigma_t2", "d_g2"):
                out[k] = torch.empty(m.n_inst, dtype=torch.float64, device=dev)
    for g in (grad_R, grad_bins, grad_R_k, grad_T):
        if g is not None:
            assert g.is_cuda and g.dtype == torch.float64 and g.is_contiguous()
    gi = GradIn(_ptr(grad_R), _ptr(grad_bins), _ptr(grad_R_k), _ptr(grad_T))
    go = GradOut(*(_ptr(out.get(k)) for k in GRAD_KEYS))
    p, oc = m.c(), o.c()
    _check(lib.sss_walk_bwd(C.byref(p), C.byref(oc), _ptr(workspace), workspace.numel(),
                            C.byref(gi), C.byref(go), _stream(stream)), "sss_walk_bwd")
    out["_workspace"] = workspace
    return out


def read_status(workspace: torch.Tensor, stream=None):
    """(status code, flag bits) left in the workspace by the last call."""
    flags = C.c_uint32(0)
    code = lib.sss_read_status(_ptr(workspace), _stream(stream), C.byref(flags))
    return code, flags.value


def last_device_status(stream=None):
    """(status code, flag bits) of the last walk, adjoint or decode call
    enqueued on `stream` (sss_last_device_status; waits for the stream)."""
    flags = C.c_uint32(0)
    code = lib.sss_last_device_status(_stream(stream), C.byref(flags))
    return code, flags.value


def philox(ctr: torch.Tensor, key: int, stream=None) -> torch.Tensor:
    """Device Philox4x32-10 blocks for int32 counters [n][4] (bit patterns)."""
    assert ctr.is_cuda and ctr.dtype == torch.int32 and ctr.shape[-1] == 4
    ctr = ctr.contiguous()
    out = torch.empty_like(ctr)
    _check(lib.sss_philox(_ptr(ctr), key, ctr.shape[0], _ptr(out), _stream(stream)), "sss_philox")
    return out


def profile_events(start=None, stop=None):
    """Record torch.cuda.Event pair around the main walk kernel of the next
    calls from this thread (None, None to stop)."""
    if start is None or stop is None:
        lib.sss_profile_events(None, None)
    else:
        lib.sss_profile_events(C.c_void_p(start.cuda_event), C.c_void_p(stop.cuda_event))


def release_plans():
    lib.sss_release_plans()


def abi_version() -> int:
    return lib.sss_abi_version()


class SSSWalk(torch.autograd.Function):
    """Differentiable forward walk: (alpha, sigma_t, g, w) -> (R, bins, R_k).

    backward runs the path-replay adjoint with the same options and seed."""

    @staticmethod
    def forward(ctx, alpha, sigma_t, g, w, template: Media, o: WalkOptions):
        m = Media(alpha.detach().contiguous(), sigma_t.detach().contiguous(),
                  g.detach().contiguous(), w.detach().contiguous(), template.n_paths,
                  template.uniform_paths, template.thickness_mm, template.n_rel,
                  template.layer2)
        r = walk(m, o)
        ctx.m, ctx.o = m, o
        return r["R"], r["bins"], r["R_k"]

    @staticmethod
    def backward(ctx, gR, gB, gK):
        f = lambda t: None if t is None else t.detach().to(torch.float64).contiguous()
        d = walk_bwd(ctx.m, ctx.o, grad_R=f(gR), grad_bins=f(gB), grad_R_k=f(gK))
        cast = lambda t: t.to(torch.float32)
        return cast(d["d_alpha"]), cast(d["d_sigma_t"]), cast(d["d_g"]), cast(d["d_w"]), \
            None, None


# ------------------------------------------------------------------ decoder --
class DecoderWeights(C.Structure):
    _fields_ = [("W", C.c_void_p * 10), ("b", C.c_void_p * 10)]


DECODER_LAYERS = ("enc0", "enc1", "enc2", "dec_r0", "dec_r1", "dec_r2",
                  "dec_t0", "dec_t1", "dec_t2", "dec_t3")


def _decoder_sigs():
    lib.sss_decoder_packed_size.argtypes = []
    lib.sss_decoder_packed_size.restype = C.c_size_t
    lib.sss_decode_workspace_size.argtypes = [C.c_int64]
    lib.sss_decode_workspace_size.restype = C.c_size_t
    lib.sss_decoder_pack.argtypes = [C.POINTER(DecoderWeights), C.c_void_p, C.c_size_t,
                                     C.c_void_p]
    lib.sss_decoder_pack.restype = C.c_int
    lib.sss_decode.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_size_t,
                               C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.sss_decode.restype = C.c_int


_decoder_sigs()


def decoder_pack(weights: dict, device="cuda", stream=None) -> torch.Tensor:
    """Packs natural-layout weights {name: (W [out][in], b [out])} (numpy or
    torch, values representable in bf16) into the library's decoder layout."""
    import numpy as np
    keep = []
    dw = DecoderWeights()
    for i, name in enumerate(DECODER_LAYERS):
        W, b = weights[name]
        Wt = torch.as_tensor(np.asarray(W, np.float32)).to(torch.bfloat16).contiguous().to(device)
        bt = torch.as_tensor(np.asarray(b, np.float32)).contiguous().to(device)
        keep += [Wt, bt]
        dw.W[i] = Wt.data_ptr()
        dw.b[i] = bt.data_ptr()
    n = lib.sss_decoder_packed_size()
    packed = torch.empty(n, dtype=torch.uint8, device=device)
    _check(lib.sss_decoder_pack(C.byref(dw), _ptr(packed), n, _stream(stream)),
           "sss_decoder_pack")
    torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
    return packed


def decode(rgb: torch.Tensor, packed: torch.Tensor, workspace: Optional[torch.Tensor] = None,
           out: Optional[dict] = None, stream=None) -> dict:
    """sss_decode: rgb float32 [T][3] CUDA -> dict alpha, g, sigma_t, w, each
    float32 [3][81*T] (band-major instances, the walk's layout)."""
    assert rgb.is_cuda and rgb.dtype == torch.float32 and rgb.is_contiguous()
    T = rgb.shape[0]
    if workspace is None:
        workspace = torch.empty(lib.sss_decode_workspace_size(T), dtype=torch.uint8,
                                device=rgb.device)
    if out is None:
        out = {k: torch.empty(3, 81 * T, dtype=torch.float32, device=rgb.device)
               for k in ("alpha", "g", "sigma_t", "w")}
    _check(lib.sss_decode(_ptr(rgb), T, _ptr(packed), _ptr(workspace), workspace.numel(),
                          _ptr(out["alpha"]), _ptr(out["g"]), _ptr(out["sigma_t"]),
                          _ptr(out["w"]), _stream(stream)), "sss_decode")
    out["_workspace"] = workspace
    return out


# ------------------------------------------------------- no-allocation walk --
NOALLOC_SCRATCH_BYTES = 16 * 1024 * 1024
lib.sss_walk_noalloc.argtypes = [C.POINTER(Params), C.POINTER(Opts), C.POINTER(Tallies),
                                 C.POINTER(C.c_uint32), C.c_void_p]
lib.sss_walk_noalloc.restype = C.c_int


def walk_noalloc(m: Media, o: WalkOptions, out: dict, stream=None, read_flags: bool = True):
    """sss_walk_noalloc: the forward walk with the library's built-in scratch
    (for callers that cannot allocate device memory).  `out` must already
    hold the output tensors (alloc_tallies).  With read_flags the call waits
    for the stream and returns (status, device flags); without, it passes no
    flag word, returns (status of the enqueue, None) at once, and the device
    status can be read later with last_device_status."""
    t = Tallies(**{k: _ptr(out.get(k)) for k in TALLY_KEYS})
    p, oc = m.c(), o.c()
    flags = C.c_uint32(0)
    code = lib.sss_walk_noalloc(C.byref(p), C.byref(oc), C.byref(t),
                                C.byref(flags) if read_flags else None, _stream(stream))
    return code, (flags.value if read_flags else None)


# --------------------------------------------------------------- LUT fit --
class Lut(C.Structure):
    _fields_ = [("R", C.c_void_p), ("p", C.c_void_p), ("na", C.c_int32), ("ng", C.c_int32),
                ("nb", C.c_int32), ("a0", C.c_float), ("da", C.c_float), ("g0", C.c_float),
                ("dg", C.c_float), ("drho", C.c_float)]


class FitOpts(C.Structure):
    _fields_ = [("K", C.c_int32), ("steps", C.c_int32), ("lr", C.c_float),
                ("lambda_R", C.c_float), ("a_lo", C.c_float), ("a_hi", C.c_float),
                ("g_lo", C.c_float), ("g_hi", C.c_float)]


lib.sss_lut_fit.argtypes = [C.POINTER(Lut), C.c_int64, C.c_void_p, C.c_int32, C.c_void_p,
                            C.c_void_p, C.POINTER(FitOpts), C.c_void_p, C.c_void_p, C.c_void_p,
                            C.c_void_p]
lib.sss_lut_fit.restype = C.c_int


def lut_fit(R_lut, p_lut, a0, da, g0, dg, drho, r_mm, P_mc, R_mc, raw, K=3, steps=1000,
            lr=1e-2, lambda_R=5.0, a_rng=(0.0, 0.999), g_rng=(0.0, 0.95), want_grad=False,
            stream=None):
    """sss_lut_fit on CUDA float32 tensors; `raw` [n_prob][4K] is updated in
    place.  Returns (loss [n_prob], grad [n_prob][4K] or None)."""
    for t in (R_lut, p_lut, r_mm, P_mc, R_mc, raw):
        assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
    na, ng, nb = p_lut.shape
    L = Lut(_ptr(R_lut), _ptr(p_lut), na, ng, nb, a0, da, g0, dg, drho)
    o = FitOpts(K, steps, lr, lambda_R, a_rng[0], a_rng[1], g_rng[0], g_rng[1])
    n = raw.shape[0]
    loss = torch.empty(n, dtype=torch.float32, device=raw.device)
    grad = torch.empty_like(raw) if want_grad else None
    _check(lib.sss_lut_fit(C.byref(L), n, _ptr(r_mm), r_mm.numel(), _ptr(P_mc), _ptr(R_mc),
                           C.byref(o), _ptr(raw), _ptr(loss), _ptr(grad), _stream(stream)),
           "sss_lut_fit")
    return loss, grad


PROBE_KINDS = {"ffma": 0, "ffma2": 1, "imad": 2, "lop3": 3, "mufu_lg2": 4, "philox": 5}


def probe(kind: str, iters: int, blocks: int, sink: torch.Tensor, stream=None) -> int:
    """Launches the issue-rate probe `kind` (see sss_probe); returns the lane
    operations it executes.  `sink` is a float32 CUDA tensor of blocks * 256."""
    k = PROBE_KINDS[kind]
    assert sink.is_cuda and sink.dtype == torch.float32 and sink.numel() >= blocks * 256
    _check(lib.sss_probe(k, iters, blocks, _ptr(sink), _stream(stream)), "sss_probe")
    return blocks * 256 * iters * lib.sss_probe_ops_per_thread_iter(k)


def selftest_bounded_wait(status: torch.Tensor, limit_cycles: int, stream=None) -> None:
    """sss_selftest_bounded_wait on a CUDA int32/uint8 tensor whose first 4
    bytes hold the status word (e.g. a decode workspace)."""
    assert status.is_cuda
    _check(lib.sss_selftest_bounded_wait(_ptr(status), limit_cycles, _stream(stream)),
           "sss_selftest_bounded_wait")
