"""Python binding of the binary Shan-Chen D2Q9 capillary library.

Argument marshalling only: every step of the method runs in the CUDA kernels
behind include/lbm.h.  PyTorch supplies device memory (its caching allocator,
through the library's allocator callback) and the stream (the current torch
stream at creation).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib as L

PRECISIONS = {"f64": L.LBM_F64, "f32": L.LBM_F32, "f16s": L.LBM_F16S}
STORAGE_DTYPE = {L.LBM_F64: np.float64, L.LBM_F32: np.float32, L.LBM_F16S: np.float16}


class _TorchDtypes(dict):
    """torch dtype of the stored populations per precision code (torch is
    imported on first use)."""
    def __missing__(self, key):
        import torch
        self.update({L.LBM_F64: torch.float64, L.LBM_F32: torch.float32, L.LBM_F16S: torch.float16})
        return self[key]


TORCH_STORAGE_DTYPE = _TorchDtypes()


class _TorchAllocator:
    """Device allocations through torch's caching allocator."""

    def __init__(self, device):
        import torch
        self._torch = torch
        self.device = device
        self.alloc = L.ALLOC_FN(self._alloc)
        self.free = L.FREE_FN(self._free)

    def _alloc(self, ctx, nbytes, stream):
        try:
            return int(self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device, int(stream or 0)))
        except Exception:  # the library turns NULL into LBM_ENOMEM
            return None

    def _free(self, ctx, ptr, nbytes, stream):
        try:
            self._torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass


def _geometry(run: dict, keep: list) -> L.Geometry:
    g = run["geom"]
    G = L.Geometry()
    G.nx, G.ny = int(g["nx"]), int(g["ny"])
    G.cap_x0, G.cap_x1 = int(g.get("cap_x0", 0)), int(g.get("cap_x1", 0))
    G.y_bot, G.y_top = int(g.get("y_bot", -1)), int(g.get("y_top", -1))
    rho = run.get("rho", (2.0, 0.04))
    G.rho_major, G.rho_minor = float(rho[0]), float(rho[1])
    if g.get("mask") is not None:
        m = np.ascontiguousarray(g["mask"], dtype=np.uint8).reshape(G.ny, G.nx)
        keep.append(m)
        G.solid_mask = m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    init = run.get("init", ("slab", 0, 0))
    kind = init[0]
    if kind == "slab":
        G.init_kind = L.LBM_INIT_SLAB
        G.x_lo, G.x_hi = float(init[1]), float(init[2])
    elif kind == "droplet":
        G.init_kind = L.LBM_INIT_DROPLET
        G.drop_cx, G.drop_cy, G.drop_r = float(init[1]), float(init[2]), float(init[3])
    elif kind == "fields":
        G.init_kind = L.LBM_INIT_FIELDS
        a = np.ascontiguousarray(init[1], dtype=np.float64).reshape(G.ny, G.nx)
        b = np.ascontiguousarray(init[2], dtype=np.float64).reshape(G.ny, G.nx)
        keep.extend([a, b])
        G.init_nA = a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        G.init_nB = b.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    else:
        raise ValueError(f"unknown init kind {kind!r}")
    return G


class Lattice:
    """One or more independent capillary runs advanced together on one GPU.

    ``runs``: a run dict or a list of them, each with ``geom`` (nx, ny,
    cap_x0, cap_x1, y_bot, y_top, optional mask), ``params`` (G, G_Aw, G_Bw,
    tau_A, tau_B; optional body, rho_bulk, alpha = (alpha_A, alpha_B) of
    Eqs. 3-5 and mass = (m_A, m_B), shared by all runs) and ``init`` (("slab", x_lo, x_hi),
    ("droplet", cx, cy, r) or ("fields", nA, nB)).
    """

    def __init__(self, runs, precision: str = "f32", log_every: int = 0, log_capacity: int = 0,
                 autotune: bool = False, tile=(128, 4), graph_chunk: int = 0, rho_ref=(0.0, 0.0),
                 stream=None, torch_allocator: bool = True, kernel=None, _handle=None):
        import torch
        lib = L.load()
        self._lib = lib
        self._torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.device = torch.cuda.current_device()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self._alloc = _TorchAllocator(self.device) if torch_allocator else None
        self._h = ctypes.c_void_p()
        if _handle is not None:
            self._h = _handle
            self.runs = None
            self._finish_init()
            return
        if isinstance(runs, dict):
            runs = [runs]
        self.runs = list(runs)
        # with an explicit kernel the tiling is set together with it after creation
        # (the creation options only know the default kernel's tilings)
        species = [(tuple(r["params"].get("alpha", (4.0 / 9.0,) * 2)), tuple(r["params"].get("mass", (1.0, 1.0))))
                   for r in self.runs]
        if any(sp != species[0] for sp in species):
            raise ValueError("alpha and mass are options of the handle: every run must give the same values")
        opt = self._options(self.runs[0]["params"], log_every, log_capacity, autotune,
                            tile if kernel is None else (0, 0), graph_chunk, rho_ref)
        keep = []
        geoms = (L.Geometry * len(self.runs))(*[_geometry(r, keep) for r in self.runs])
        n = len(self.runs)
        G = (ctypes.c_double * n)(*[float(r["params"]["G"]) for r in self.runs])
        wall = (ctypes.c_double * (2 * n))(*[float(v) for r in self.runs
                                             for v in (r["params"].get("G_Aw", 0.0), r["params"].get("G_Bw", 0.0))])
        tA = (ctypes.c_double * n)(*[float(r["params"]["tau_A"]) for r in self.runs])
        tB = (ctypes.c_double * n)(*[float(r["params"]["tau_B"]) for r in self.runs])
        with torch.cuda.device(self.device):
            L.check(lib.lbm_create_batch(n, geoms, G, wall, tA, tB, ctypes.byref(opt), ctypes.byref(self._h)),
                    "lbm_create_batch")
        self._finish_init()
        if kernel is not None:   # (kernel, depth)
            try:
                self.schedule = (int(tile[0]), int(tile[1]), int(kernel[0]), int(kernel[1]))
            except Exception:
                self.close()
                raise

    def _options(self, prm, log_every, log_capacity, autotune, tile, graph_chunk, rho_ref) -> L.Options:
        opt = L.Options()
        self._lib.lbm_default_options(ctypes.byref(opt))
        opt.precision = self.precision
        opt.log_every = int(log_every)
        opt.log_capacity = int(log_capacity or (max(1, 1 << 16) if log_every else 0))
        opt.autotune = int(bool(autotune))
        opt.tile_w, opt.tile_h = int(tile[0]), int(tile[1])
        opt.graph_chunk = int(graph_chunk)
        opt.rho_ref[0], opt.rho_ref[1] = float(rho_ref[0]), float(rho_ref[1])
        opt.rho_bulk = float(prm.get("rho_bulk", 2.0))
        body = prm.get("body", (0.0, 0.0))
        opt.body[0], opt.body[1] = float(body[0]), float(body[1])
        alpha = prm.get("alpha", (4.0 / 9.0, 4.0 / 9.0))
        mass = prm.get("mass", (1.0, 1.0))
        opt.alpha[0], opt.alpha[1] = float(alpha[0]), float(alpha[1])
        opt.molecular_mass[0], opt.molecular_mass[1] = float(mass[0]), float(mass[1])
        if self._alloc is not None:
            opt.alloc, opt.free = self._alloc.alloc, self._alloc.free
        opt.stream = ctypes.c_void_p(int(self.stream.cuda_stream))
        self._opt = opt
        return opt

    def _finish_init(self):
        self.nruns = int(self._lib.lbm_num_runs(self._h))
        self.shapes = []
        for r in range(self.nruns):
            info = self.run_info(r)
            self.shapes.append((info.ny, info.nx))

    # ---- lifecycle -----------------------------------------------------
    def close(self):
        if self._h:
            self._lib.lbm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- stepping ------------------------------------------------------
    def step(self, n: int = 1) -> None:
        L.check(self._lib.lbm_step(self._h, int(n)), "lbm_step")

    def sync(self) -> None:
        L.check(self._lib.lbm_sync(self._h), "lbm_sync")

    @property
    def t(self) -> int:
        return int(self._lib.lbm_time(self._h))

    def status(self) -> int:
        return int(self._lib.lbm_status(self._h))

    def run_info(self, run: int = 0) -> L.RunInfo:
        info = L.RunInfo()
        L.check(self._lib.lbm_run_info_get(self._h, int(run), ctypes.byref(info)), "lbm_run_info_get")
        return info

    @property
    def tiling(self):
        w, h = ctypes.c_int(), ctypes.c_int()
        L.check(self._lib.lbm_get_tiling(self._h, ctypes.byref(w), ctypes.byref(h)), "lbm_get_tiling")
        return int(w.value), int(h.value)

    @tiling.setter
    def tiling(self, wh):
        L.check(self._lib.lbm_set_tiling(self._h, int(wh[0]), int(wh[1])), "lbm_set_tiling")

    @property
    def schedule(self):
        """(tile_w, tile_h, kernel, depth); kernel is one of the LBM_KERNEL_*
        variants of include/lbm.h (0 register pull, 1 cp.async stages, 2 TMA
        ring, 3 pipelined, 4 species split, 5 L2 prefetch, 6 shared-memory
        staged, 7 column pair, 8 node tile, 9 bidirectional, 10 persistent
        ring, 11 bidirectional compiled at run time for the run's grid)."""
        v = [ctypes.c_int() for _ in range(4)]
        L.check(self._lib.lbm_get_schedule(self._h, *[ctypes.byref(x) for x in v]), "lbm_get_schedule")
        return tuple(int(x.value) for x in v)

    @schedule.setter
    def schedule(self, s):
        L.check(self._lib.lbm_set_schedule(self._h, int(s[0]), int(s[1]), int(s[2]), int(s[3])), "lbm_set_schedule")

    def tuning(self):
        """The autotuner's finalists: [((tile_w, tile_h, kernel, depth),
        ms per step on back-to-back steps), ...]; empty before tuning."""
        n = ctypes.c_int()
        L.check(self._lib.lbm_get_tuning(self._h, 0, None, None, ctypes.byref(n)), "lbm_get_tuning")
        k = n.value
        sched = (ctypes.c_int * max(1, 4 * k))()
        ms = (ctypes.c_float * max(1, k))()
        L.check(self._lib.lbm_get_tuning(self._h, k, sched, ms, ctypes.byref(n)), "lbm_get_tuning")
        return [(tuple(sched[4 * j:4 * j + 4]), float(ms[j])) for j in range(k)]

    # ---- observables ---------------------------------------------------
    def _pair(self, fn, run, device, name):
        ny, nx = self.shapes[run]
        if device:
            t = self._torch
            a = t.empty((ny, nx), dtype=t.float64, device=f"cuda:{self.device}")
            b = t.empty_like(a)
            L.check(fn(self._h, int(run), ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), 1), name)
            return a, b
        a = np.empty((ny, nx), dtype=np.float64)
        b = np.empty((ny, nx), dtype=np.float64)
        L.check(fn(self._h, int(run), a.ctypes.data_as(ctypes.c_void_p), b.ctypes.data_as(ctypes.c_void_p), 0), name)
        return a, b

    def densities(self, run: int = 0, device: bool = False):
        """(n_A, n_B) at time t, FP64 [ny, nx]."""
        return self._pair(self._lib.lbm_densities, run, device, "lbm_densities")

    def velocity(self, run: int = 0, device: bool = False):
        """Whole-fluid velocity (u_x, u_y) at time t, FP64 [ny, nx]."""
        return self._pair(self._lib.lbm_velocity, run, device, "lbm_velocity")

    def interface(self, run: int = 0) -> np.ndarray:
        """[z_bulk, z_prec_bottom, z_prec_top] measured from cap_x0."""
        zb = ctypes.c_double()
        zp = (ctypes.c_double * 2)()
        L.check(self._lib.lbm_interface_positions(self._h, int(run), ctypes.byref(zb), zp), "lbm_interface_positions")
        return np.array([zb.value, zp[0], zp[1]])

    def mass(self, run: int = 0) -> np.ndarray:
        M = (ctypes.c_double * 2)()
        L.check(self._lib.lbm_mass(self._h, int(run), M), "lbm_mass")
        return np.array([M[0], M[1]])

    def log(self, run: int = 0) -> np.ndarray:
        """Records (t, z_bulk, z_prec_bottom, z_prec_top, M_A, M_B), oldest first."""
        cap = int(self._opt.log_capacity) if getattr(self, "_opt", None) else 1 << 16
        rec = np.zeros((cap, 6))
        n = ctypes.c_int()
        L.check(self._lib.lbm_get_log(self._h, int(run), rec.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), cap,
                                      ctypes.byref(n)), "lbm_get_log")
        return rec[: n.value].copy()

    def populations(self, run: int = 0) -> np.ndarray:
        """Stored populations [2, 9, ny, nx] (FP16S: f - w_i rho_ref as stored)."""
        ny, nx = self.shapes[run]
        out = np.empty((2, 9, ny, nx), dtype=STORAGE_DTYPE[self.precision])
        L.check(self._lib.lbm_populations(self._h, int(run), out.ctypes.data_as(ctypes.c_void_p), 0), "lbm_populations")
        return out

    # ---- column windows (x-slab halo exchange) ---------------------------
    def get_columns(self, x0: int, ncols: int, run: int = 0, out=None):
        """Populations of columns [x0, x0 + ncols): a device tensor
        [2, 9, ny, ncols] in the storage dtype (into `out` if given)."""
        ny, _ = self.shapes[run]
        if out is None:
            out = self._torch.empty((2, 9, ny, int(ncols)), dtype=TORCH_STORAGE_DTYPE[self.precision],
                                    device=f"cuda:{self.device}")
        L.check(self._lib.lbm_get_columns(self._h, int(run), int(x0), int(ncols), ctypes.c_void_p(out.data_ptr()), 1),
                "lbm_get_columns")
        return out

    def set_columns(self, x0: int, buf, run: int = 0) -> None:
        """Overwrites columns [x0, x0 + ncols) from a contiguous device tensor
        [2, 9, ny, ncols] in the storage dtype."""
        assert buf.is_contiguous() and buf.is_cuda
        L.check(self._lib.lbm_set_columns(self._h, int(run), int(x0), int(buf.shape[-1]),
                                          ctypes.c_void_p(buf.data_ptr()), 1), "lbm_set_columns")

    # ---- checkpoints ---------------------------------------------------
    def save(self, path: str) -> None:
        L.check(self._lib.lbm_save(self._h, str(path).encode()), "lbm_save")

    @classmethod
    def load(cls, path: str, stream=None, torch_allocator: bool = True) -> "Lattice":
        import torch
        lib = L.load()
        self = cls.__new__(cls)
        self._lib = lib
        self._torch = torch
        self.device = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._alloc = _TorchAllocator(self.device) if torch_allocator else None
        opt = L.Options()
        lib.lbm_default_options(ctypes.byref(opt))
        if self._alloc is not None:
            opt.alloc, opt.free = self._alloc.alloc, self._alloc.free
        opt.stream = ctypes.c_void_p(int(self.stream.cuda_stream))
        h = ctypes.c_void_p()
        L.check(lib.lbm_load(str(path).encode(), ctypes.byref(opt), ctypes.byref(h)), "lbm_load")
        self._h = h
        self.runs = None
        info = L.RunInfo()
        lib.lbm_run_info_get(h, 0, ctypes.byref(info))
        self.precision = info.precision
        self._opt = None
        self._finish_init()
        return self


def run_from_workload(run: dict, rho=(2.0, 0.04)) -> dict:
    """Normalises a workloads run dict for Lattice (adds the slab/droplet densities)."""
    out = dict(run)
    out.setdefault("rho", rho)
    return out
