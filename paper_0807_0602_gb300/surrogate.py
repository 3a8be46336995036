"""Surrogate network that proposes wall couplings for a target contact angle.

The paper maps wall coupling to contact angle only a posteriori, by running
the model (Model section, after Eq. 11); this module learns that map (and the
Washburn and precursor prefactors) from runs of the lattice model and inverts
it.  Every proposal is checked by running the lattice model, which stays the
judge and the fallback.

The network and its training run in the CUDA kernels behind include/mlp.h;
this module marshals arguments (torch tensors for device memory) and holds
the host-side data handling: input/target normalisation and the candidate
search that inverts the network along a one-parameter coupling family.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib as L

N_PARAMS = 34307
N_IN, N_OUT = 6, 3

MLP_SIGNATURES = {
    "mlp_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_float), ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_void_p)]),
    "mlp_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]),
    "mlp_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]),
    "mlp_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "mlp_gradients": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_void_p]),
    "mlp_train_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                      ctypes.c_float, ctypes.c_void_p]),
    "mlp_step_count": (ctypes.c_int64, [ctypes.c_void_p]),
    "mlp_destroy": (None, [ctypes.c_void_p]),
}


def _load():
    lib = L.load()
    for name, (res, args) in MLP_SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def _check(code, where):
    if code != 0:
        raise RuntimeError(f"{where} failed with code {code}")


def init_params(seed: int) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases (PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for a, b in ((6, 128), (128, 128), (128, 128), (128, 3)):
        lim = 1.0 / np.sqrt(a)
        parts.append(rng.uniform(-lim, lim, size=a * b))
        parts.append(np.zeros(b))
    return np.concatenate(parts).astype(np.float32)


class Network:
    """Handle on the device network (FP32 master weights, bf16 GEMM operands)."""

    def __init__(self, max_batch: int = 4096, params: np.ndarray | None = None, stream=None):
        import torch
        self._torch = torch
        self._lib = _load()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.max_batch = int(max_batch)
        self._h = ctypes.c_void_p()
        p = None
        if params is not None:
            self._p = np.ascontiguousarray(params, dtype=np.float32)
            assert self._p.size == N_PARAMS
            p = self._p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        _check(self._lib.mlp_create(self.max_batch, p, ctypes.c_void_p(int(self.stream.cuda_stream)),
                                    ctypes.byref(self._h)), "mlp_create")

    def close(self):
        if self._h:
            self._lib.mlp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def params(self) -> np.ndarray:
        out = np.empty(N_PARAMS, dtype=np.float32)
        _check(self._lib.mlp_get_params(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), "mlp_get_params")
        return out

    @params.setter
    def params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(self._lib.mlp_set_params(self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), "mlp_set_params")

    @property
    def steps(self) -> int:
        return int(self._lib.mlp_step_count(self._h))

    def _dev(self, a, cols):
        t = self._torch
        if not isinstance(a, t.Tensor):
            a = t.as_tensor(np.asarray(a, dtype=np.float32))
        a = a.to(device="cuda", dtype=t.float32).contiguous()
        assert a.dim() == 2 and a.shape[1] == cols
        return a

    def forward(self, x):
        x = self._dev(x, N_IN)
        y = self._torch.empty((x.shape[0], N_OUT), dtype=self._torch.float32, device="cuda")
        _check(self._lib.mlp_forward(self._h, ctypes.c_void_p(x.data_ptr()), x.shape[0], ctypes.c_void_p(y.data_ptr())),
               "mlp_forward")
        return y

    def gradients(self, x, t):
        x, t = self._dev(x, N_IN), self._dev(t, N_OUT)
        g = self._torch.empty(N_PARAMS, dtype=self._torch.float32, device="cuda")
        loss = self._torch.empty(1, dtype=self._torch.float32, device="cuda")
        _check(self._lib.mlp_gradients(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()), x.shape[0],
                                       ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(loss.data_ptr())), "mlp_gradients")
        return g, loss

    def train_step(self, x, t, lr: float):
        x, t = self._dev(x, N_IN), self._dev(t, N_OUT)
        loss = self._torch.empty(1, dtype=self._torch.float32, device="cuda")
        _check(self._lib.mlp_train_step(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                        x.shape[0], float(lr), ctypes.c_void_p(loss.data_ptr())), "mlp_train_step")
        return loss


class Normalizer:
    """Per-column affine map to zero mean, unit spread (host-side data handling)."""

    def __init__(self, data: np.ndarray):
        data = np.asarray(data, dtype=np.float64)
        self.mean = data.mean(axis=0)
        self.scale = np.where(data.std(axis=0) > 0, data.std(axis=0), 1.0)

    def fwd(self, a):
        return (np.asarray(a, dtype=np.float64) - self.mean) / self.scale

    def inv(self, a):
        return np.asarray(a, dtype=np.float64) * self.scale + self.mean


class Surrogate:
    """Inputs (G_Aw, G_Bw, G_AB, tau_A, tau_B, H) -> targets (cos theta,
    Washburn prefactor, precursor prefactor), trained with the device kernels."""

    def __init__(self, X: np.ndarray, T: np.ndarray, seed: int = 0, max_batch: int = 4096):
        self.xn = Normalizer(X)
        self.tn = Normalizer(T)
        self.net = Network(max_batch=max_batch, params=init_params(seed))

    def fit(self, X, T, steps: int = 2000, lr: float = 2e-3, batch: int = 512, seed: int = 0):
        import torch
        rng = np.random.Generator(np.random.PCG64(seed))
        Xd = torch.as_tensor(self.xn.fwd(X), dtype=torch.float32, device="cuda")
        Td = torch.as_tensor(self.tn.fwd(T), dtype=torch.float32, device="cuda")
        n = Xd.shape[0]
        losses = []
        for s in range(steps):
            idx = torch.as_tensor(rng.choice(n, size=min(batch, n), replace=False), device="cuda")
            losses.append(self.net.train_step(Xd[idx], Td[idx], lr))
        return torch.cat(losses).cpu().numpy()

    def predict(self, X) -> np.ndarray:
        y = self.net.forward(self.xn.fwd(X)).cpu().numpy()
        return self.tn.inv(y)

    def propose(self, targets_cos, fixed, family: str = "A", lo: float = -0.6, hi: float = 0.6,
                n_cand: int = 1201, other: float = 0.0) -> np.ndarray:
        """For each target cos(theta), the coupling on the candidate grid of the
        one-parameter family (family "A": G_Aw varies, G_Bw = other; "B": the
        reverse) whose predicted cos(theta) is closest.  ``fixed`` =
        (G_AB, tau_A, tau_B, H).  Returns [n_targets, 2] couplings (G_Aw, G_Bw)."""
        grid = np.linspace(lo, hi, n_cand)
        X = np.zeros((n_cand, 6))
        if family == "A":
            X[:, 0] = grid
            X[:, 1] = other
        else:
            X[:, 1] = grid
            X[:, 0] = other
        X[:, 2:] = np.asarray(fixed, dtype=np.float64)[None, :]
        cos_pred = self.predict(X)[:, 0]
        out = np.zeros((len(targets_cos), 2))
        out[:, 1 if family == "A" else 0] = other
        for j, c in enumerate(targets_cos):
            k = int(np.argmin(np.abs(cos_pred - c)))
            out[j, 0 if family == "A" else 1] = grid[k]
        return out
