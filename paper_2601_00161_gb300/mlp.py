"""ctypes binding of include/esp_mlp.h: the selector's 3-layer perceptron, trained and
evaluated by the library's CUDA kernels (argument marshalling only)."""

from __future__ import annotations

import ctypes

import numpy as np

from . import LIB_PATH

EXPORTS = (
    "esp_mlp_n_params", "esp_mlp_create", "esp_mlp_forward", "esp_mlp_loss_grad",
    "esp_mlp_adam", "esp_mlp_get_params", "esp_mlp_set_params", "esp_mlp_destroy",
    "esp_mlp_last_error",
)


class MLPError(RuntimeError):
    pass


def _load():
    lib = ctypes.CDLL(LIB_PATH)
    vp, ci, cf = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
    fptr = ctypes.POINTER(ctypes.c_float)
    sig = {
        "esp_mlp_n_params": (ci, [ci, ci, ci]),
        "esp_mlp_create": (ci, [ctypes.POINTER(vp), ci, ci, ci, ci, fptr, vp]),
        "esp_mlp_forward": (ci, [vp, vp, ci, vp]),
        "esp_mlp_loss_grad": (ci, [vp, vp, vp, ci, vp, vp]),
        "esp_mlp_adam": (ci, [vp, cf, cf, cf, cf]),
        "esp_mlp_get_params": (ci, [vp, fptr]),
        "esp_mlp_set_params": (ci, [vp, fptr]),
        "esp_mlp_destroy": (ci, [vp]),
        "esp_mlp_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def _check(code):
    if code != 0:
        m = _lib.esp_mlp_last_error()
        raise MLPError(f"esp_mlp error {code}: {m.decode() if m else ''}")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _fp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


# ---- the C ABI, same names ---------------------------------------------------------------
def esp_mlp_n_params(n_in, n_hidden, n_out) -> int:
    return _lib.esp_mlp_n_params(int(n_in), int(n_hidden), int(n_out))


def esp_mlp_create(n_in, n_hidden, n_out, max_batch, params: np.ndarray, stream=None):
    h = ctypes.c_void_p()
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(_lib.esp_mlp_create(ctypes.byref(h), int(n_in), int(n_hidden), int(n_out),
                               int(max_batch), _fp(p), ctypes.c_void_p(stream) if stream else None))
    return h


def esp_mlp_forward(net, x, batch, y):
    _check(_lib.esp_mlp_forward(net, _ptr(x), int(batch), _ptr(y)))


def esp_mlp_loss_grad(net, x, t, batch, loss, grad=None):
    _check(_lib.esp_mlp_loss_grad(net, _ptr(x), _ptr(t), int(batch), _ptr(loss), _ptr(grad)))


def esp_mlp_adam(net, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    _check(_lib.esp_mlp_adam(net, float(lr), float(beta1), float(beta2), float(eps)))


def esp_mlp_get_params(net, out: np.ndarray):
    _check(_lib.esp_mlp_get_params(net, _fp(out)))


def esp_mlp_set_params(net, params: np.ndarray):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(_lib.esp_mlp_set_params(net, _fp(p)))


def esp_mlp_destroy(net):
    _lib.esp_mlp_destroy(net)


def esp_mlp_last_error() -> str:
    m = _lib.esp_mlp_last_error()
    return m.decode() if m else ""


class MLP:
    """Owns an esp_mlp_t; batches are torch CUDA float32 tensors."""

    def __init__(self, n_in, n_hidden, n_out, max_batch, params=None, seed=0, stream=None):
        if min(n_in, n_hidden, n_out, max_batch) < 1:
            raise MLPError("sizes must be positive")
        self.n_in, self.n_hidden, self.n_out, self.max_batch = n_in, n_hidden, n_out, max_batch
        self.n_params = esp_mlp_n_params(n_in, n_hidden, n_out)
        if params is None:
            params = self.init_params(seed)
        self.handle = esp_mlp_create(n_in, n_hidden, n_out, max_batch, params, stream)

    def init_params(self, seed):
        """Glorot-uniform weights, zero biases (host side, seeded)."""
        rng = np.random.default_rng(seed)
        out = []
        for fan_in, fan_out in ((self.n_in, self.n_hidden), (self.n_hidden, self.n_hidden),
                                (self.n_hidden, self.n_out)):
            a = np.sqrt(6.0 / (fan_in + fan_out))
            out += [rng.uniform(-a, a, size=fan_out * fan_in), np.zeros(fan_out)]
        return np.concatenate(out).astype(np.float32)

    def params(self) -> np.ndarray:
        a = np.empty(self.n_params, dtype=np.float32)
        esp_mlp_get_params(self.handle, a)
        return a

    def set_params(self, p):
        esp_mlp_set_params(self.handle, p)

    def forward(self, x):
        import torch

        y = torch.empty((x.shape[0], self.n_out), dtype=torch.float32, device="cuda")
        esp_mlp_forward(self.handle, x.contiguous(), x.shape[0], y)
        return y

    def loss_grad(self, x, t, want_grad=False):
        import torch

        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        g = torch.empty(self.n_params, dtype=torch.float32, device="cuda") if want_grad else None
        esp_mlp_loss_grad(self.handle, x.contiguous(), t.contiguous(), x.shape[0], loss, g)
        return loss, g

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        esp_mlp_adam(self.handle, lr, beta1, beta2, eps)

    def close(self):
        if getattr(self, "handle", None):
            esp_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
