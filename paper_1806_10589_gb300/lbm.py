"""ctypes binding of libgb300lbm.so (include/lbm.h): argument marshalling only.

Every computation runs in the CUDA library.  The module-level functions carry
the C names and signatures; `Lattice` is a thin owner of one lbm_ctx that
marshals numpy arrays.  Importing works without a GPU; the first call that
needs the library raises if libgb300lbm.so has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# GB300_LBM_LIB selects another build of the same library (e.g. a tuning variant)
LIB_PATH = os.environ.get("GB300_LBM_LIB") or os.path.join(_HERE, "libgb300lbm.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSUPPORTED, LBM_EUNSTABLE, LBM_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
LBM_MODEL_BGK, LBM_MODEL_MRT = 0, 1
LBM_PREC_FP64, LBM_PREC_FP32, LBM_PREC_FP16DEV, LBM_PREC_BF16DEV = 0, 1, 2, 3
LBM_BATCH_GRAPH, LBM_BATCH_GRAPH_CAPPED, LBM_BATCH_PERSISTENT, LBM_BATCH_PERSISTENT_CAPPED = 0, 1, 2, 3
LBM_BATCH_AA, LBM_BATCH_AA_CAPPED = 4, 5
LBM_BATCH_NCONFIG = 6
BATCH_CONFIGS = ("graph", "graph-capped", "persistent", "persistent-capped", "aa", "aa-capped")
LBM_FACE_ZMIN, LBM_FACE_ZMAX = 4, 5
PRECISIONS = {"fp64": LBM_PREC_FP64, "fp32": LBM_PREC_FP32, "fp16dev": LBM_PREC_FP16DEV,
              "bf16dev": LBM_PREC_BF16DEV}
MODELS = {"bgk": LBM_MODEL_BGK, "mrt": LBM_MODEL_MRT}
STATUS_NAMES = {0: "LBM_OK", -1: "LBM_EINVAL", -2: "LBM_ENOMEM", -3: "LBM_ECUDA",
                -4: "LBM_EUNSUPPORTED", -5: "LBM_EUNSTABLE", -6: "LBM_ETIMEOUT"}

_P = C.c_void_p
_DP = C.POINTER(C.c_double)
_I64P = C.POINTER(C.c_int64)
_FP = C.POINTER(C.c_float)

# name -> (restype, argtypes), the exact list declared in include/lbm.h
SIGNATURES = {
    "lbm_create": (C.c_int, [C.POINTER(C.c_uint8), C.c_int, C.c_int, C.c_int, C.c_double, C.c_int,
                             C.c_int, C.POINTER(_P)]),
    "lbm_set_flux_bc": (C.c_int, [_P, C.c_int, C.c_double]),
    "lbm_set_pressure_bc": (C.c_int, [_P, C.c_int, C.c_double]),
    "lbm_set_stream": (C.c_int, [_P, _P]),
    "lbm_set_kernel": (C.c_int, [_P, C.c_int]),
    "lbm_step": (C.c_int, [_P, C.c_int]),
    "lbm_get_flux": (C.c_int, [_P, C.c_int, _DP, _DP]),
    "lbm_get_monitors": (C.c_int, [_P, _DP, _DP, _DP, _DP]),
    "lbm_steady_residual": (C.c_int, [_P, _DP]),
    "lbm_get_fields": (C.c_int, [_P, _DP, _DP, _DP, _DP]),
    "lbm_get_fields_device": (C.c_int, [_P, _P, _P]),
    "lbm_set_fields": (C.c_int, [_P, _DP, _DP, _DP, _DP]),
    "lbm_get_distributions": (C.c_int, [_P, _DP]),
    "lbm_set_distributions": (C.c_int, [_P, _DP]),
    "lbm_get_info": (C.c_int, [_P, _I64P, _I64P, _I64P, _I64P]),
    "lbm_time_kernels": (C.c_int, [_P, C.c_int, _FP, _FP]),
    "lbm_inlet_density_noalloc": (C.c_int, [_P, _P]),
    "lbm_destroy": (C.c_int, [_P]),
    "lbm_last_error": (C.c_char_p, [_P]),
    "lbm_batch_create": (C.c_int, [C.c_int, C.POINTER(C.POINTER(C.c_uint8)), C.POINTER(C.c_int), C.c_double,
                                   C.c_int, C.c_int, C.POINTER(_P)]),
    "lbm_batch_set_flux_bc": (C.c_int, [_P, C.c_int, C.c_double]),
    "lbm_batch_set_stream": (C.c_int, [_P, _P]),
    "lbm_batch_step": (C.c_int, [_P, C.c_int]),
    "lbm_batch_get_flux": (C.c_int, [_P, C.c_int, C.c_int, _DP, _DP]),
    "lbm_batch_get_distributions": (C.c_int, [_P, C.c_int, _DP]),
    "lbm_batch_set_distributions": (C.c_int, [_P, C.c_int, _DP]),
    "lbm_batch_get_fields": (C.c_int, [_P, C.c_int, _DP, _DP, _DP, _DP]),
    "lbm_batch_get_info": (C.c_int, [_P, _I64P, _I64P, _I64P]),
    "lbm_batch_time_step": (C.c_int, [_P, C.c_int, _FP]),
    "lbm_batch_set_config": (C.c_int, [_P, C.c_int]),
    "lbm_batch_autotune": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int), _FP]),
    "lbm_batch_check_barrier": (C.c_int, [_P, C.c_double, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "lbm_batch_destroy": (C.c_int, [_P]),
    "lbm_batch_last_error": (C.c_char_p, [_P]),
    "lbm_color_create": (C.c_int, [C.POINTER(C.c_uint8), C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                   C.c_double, C.c_double, C.c_int, C.POINTER(_P)]),
    "lbm_color_set_stream": (C.c_int, [_P, _P]),
    "lbm_color_set_flux_bc": (C.c_int, [_P, C.c_double, C.c_double]),
    "lbm_color_set_phase": (C.c_int, [_P, _DP, _DP]),
    "lbm_color_set_state": (C.c_int, [_P, _DP, _DP, _DP]),
    "lbm_color_get_state": (C.c_int, [_P, _DP, _DP, _DP]),
    "lbm_color_step": (C.c_int, [_P, C.c_int]),
    "lbm_color_get_fields": (C.c_int, [_P, _DP, _DP, _DP, _DP, _DP]),
    "lbm_color_get_flux": (C.c_int, [_P, C.c_int, _DP, _DP]),
    "lbm_color_destroy": (C.c_int, [_P]),
    "lbm_color_last_error": (C.c_char_p, [_P]),
    "lbm_wsnet_create": (C.c_int, [C.c_int, C.c_int, C.POINTER(_P)]),
    "lbm_wsnet_num_params": (C.c_int, [_P, _I64P]),
    "lbm_wsnet_set_stream": (C.c_int, [_P, _P]),
    "lbm_wsnet_set_params": (C.c_int, [_P, _FP]),
    "lbm_wsnet_get_params": (C.c_int, [_P, _FP]),
    "lbm_wsnet_loss_grad": (C.c_int, [_P, C.POINTER(C.c_uint8), _FP, C.c_int, C.c_int, C.c_int, C.c_int, _DP,
                                      _FP]),
    "lbm_wsnet_train": (C.c_int, [_P, C.POINTER(C.c_uint8), _FP, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                  C.c_int, C.c_float, C.POINTER(C.c_int), _FP]),
    "lbm_wsnet_predict": (C.c_int, [_P, C.POINTER(C.c_uint8), C.c_int, C.c_int, C.c_int, _FP]),
    "lbm_wsnet_release_buffers": (C.c_int, [_P]),
    "lbm_wsnet_destroy": (C.c_int, [_P]),
    "lbm_wsnet_last_error": (C.c_char_p, [_P]),
    "lbm_conv3d_bf16": (C.c_int, [C.c_int, _P, _P, _P, _FP, C.c_int, _P, C.c_int, C.c_int, C.c_int, C.c_int,
                                  C.c_int, C.c_int, _P]),
    "lbm_conv3d_bf16_time": (C.c_int, [C.c_int, _P, _P, _P, _FP, C.c_int, _P, C.c_int, C.c_int, C.c_int, C.c_int,
                                       C.c_int, C.c_int, C.c_int, _FP, _P]),
}

_lib = None


class LBMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def load_library(path: str = LIB_PATH):
    """Load libgb300lbm.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libgb300lbm.so not built (%s); run __graft_entry__.build()" % path)
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a, ctype):
    return None if a is None else a.ctypes.data_as(C.POINTER(ctype))


def _make_raw(name):
    def raw(*args):
        return getattr(load_library(), name)(*args)
    raw.__name__ = name
    raw.__doc__ = "Raw C call %s (see include/lbm.h)." % name
    return raw


for _n in SIGNATURES:
    globals()[_n] = _make_raw(_n)


class Lattice:
    """One solver context.  mask: uint8 [nz][ny][nx], 1 = solid."""

    def __init__(self, mask, tau, model="mrt", precision="fp64", stream=None):
        lib = load_library()
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        if mask.ndim != 3:
            raise ValueError("mask must be 3-D [z][y][x]")
        self.nz, self.ny, self.nx = mask.shape
        self.shape = mask.shape
        self.mask = mask
        h = _P()
        st = lib.lbm_create(_ptr(mask, C.c_uint8), self.nx, self.ny, self.nz, float(tau),
                            MODELS[model] if isinstance(model, str) else int(model),
                            PRECISIONS[precision] if isinstance(precision, str) else int(precision),
                            C.byref(h))
        if st != LBM_OK:
            raise LBMError(st, lib.lbm_last_error(None).decode())
        self._h = h
        self._lib = lib
        if stream is not None:
            self.set_stream(stream)

    # -- plumbing
    def _check(self, st):
        if st != LBM_OK:
            raise LBMError(st, self._lib.lbm_last_error(self._h).decode())
        return st

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- calls
    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, an integer cudaStream_t handle, or None."""
        h = getattr(stream, "cuda_stream", stream)
        self._check(self._lib.lbm_set_stream(self._h, _P(h) if h else None))

    def set_flux_bc(self, Q, face=LBM_FACE_ZMIN):
        self._check(self._lib.lbm_set_flux_bc(self._h, face, float(Q)))

    def set_pressure_bc(self, face, rho):
        self._check(self._lib.lbm_set_pressure_bc(self._h, face, float(rho)))

    def set_kernel(self, variant):
        """Step-kernel variant: 0 per-node (default), 1 pipelined 256-node tiles,
        2 pipelined 128, 3 AA pattern (one buffer, FP64/FP32)."""
        self._check(self._lib.lbm_set_kernel(self._h, int(variant)))

    def step(self, n=1):
        self._check(self._lib.lbm_step(self._h, int(n)))

    def get_flux(self, face=LBM_FACE_ZMIN):
        q, r = C.c_double(), C.c_double()
        self._check(self._lib.lbm_get_flux(self._h, face, C.byref(q), C.byref(r)))
        return q.value, r.value

    def monitors(self, raise_unstable=True):
        v = [C.c_double() for _ in range(4)]
        st = self._lib.lbm_get_monitors(self._h, *[C.byref(x) for x in v])
        if st != LBM_OK and (raise_unstable or st != LBM_EUNSTABLE):
            self._check(st)
        out = dict(zip(("mass", "q_in", "q_out", "u_max"), (x.value for x in v)))
        out["status"] = st
        return out

    def steady_residual(self):
        """Section 3.1 criterion against the snapshot of the previous call
        (+inf on the first call)."""
        r = C.c_double()
        self._check(self._lib.lbm_steady_residual(self._h, C.byref(r)))
        return r.value

    def fields(self):
        arrs = [np.empty(self.shape) for _ in range(4)]
        self._check(self._lib.lbm_get_fields(self._h, *[_ptr(a, C.c_double) for a in arrs]))
        return tuple(arrs)

    def fields_device(self, rho, u):
        """rho, u: torch float32 CUDA tensors of nx*ny*nz and 3*nx*ny*nz elements."""
        self._check(self._lib.lbm_get_fields_device(self._h, _P(rho.data_ptr()), _P(u.data_ptr())))

    def set_fields(self, rho=None, ux=None, uy=None, uz=None):
        cv = [None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(self.shape)
              for a in (rho, ux, uy, uz)]
        self._check(self._lib.lbm_set_fields(self._h, *[_ptr(a, C.c_double) for a in cv]))

    def distributions(self):
        f = np.empty((19,) + self.shape)
        self._check(self._lib.lbm_get_distributions(self._h, _ptr(f, C.c_double)))
        return f

    def set_distributions(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        if f.shape != (19,) + self.shape:
            raise ValueError("f must have shape (19,) + mask.shape")
        self._check(self._lib.lbm_set_distributions(self._h, _ptr(f, C.c_double)))

    def info(self):
        v = [C.c_int64() for _ in range(4)]
        self._check(self._lib.lbm_get_info(self._h, *[C.byref(x) for x in v]))
        return dict(zip(("n_pore", "a_in", "a_out", "steps"), (x.value for x in v)))

    def inlet_density_noalloc(self, rho_in_device):
        """rho_in of Eq. (potential) for the current state into a caller-owned
        device double (e.g. a torch float64 CUDA tensor), allocating nothing."""
        ptr = rho_in_device.data_ptr() if hasattr(rho_in_device, "data_ptr") else int(rho_in_device)
        self._check(self._lib.lbm_inlet_density_noalloc(self._h, _P(ptr)))

    def time_kernels(self, n):
        a, b = C.c_float(), C.c_float()
        self._check(self._lib.lbm_time_kernels(self._h, int(n), C.byref(a), C.byref(b)))
        return a.value, b.value


class Batch:
    """A batched ensemble (lbm_batch_*): masks is a list of uint8 [z][y][x] arrays."""

    def __init__(self, masks, tau, model="mrt", precision="fp16dev", stream=None):
        lib = load_library()
        self._masks = [np.ascontiguousarray(m, dtype=np.uint8) for m in masks]
        n = len(self._masks)
        ptrs = (C.POINTER(C.c_uint8) * n)(*[_ptr(m, C.c_uint8) for m in self._masks])
        dims = (C.c_int * (3 * n))(*[v for m in self._masks for v in (m.shape[2], m.shape[1], m.shape[0])])
        h = _P()
        st = lib.lbm_batch_create(n, ptrs, dims, float(tau),
                                  MODELS[model] if isinstance(model, str) else int(model),
                                  PRECISIONS[precision] if isinstance(precision, str) else int(precision),
                                  C.byref(h))
        if st != LBM_OK:
            raise LBMError(st, lib.lbm_batch_last_error(None).decode())
        self._h, self._lib = h, lib
        if stream is not None:
            hs = getattr(stream, "cuda_stream", stream)
            self._check(lib.lbm_batch_set_stream(h, _P(hs) if hs else None))

    def _check(self, st):
        if st != LBM_OK:
            raise LBMError(st, self._lib.lbm_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __len__(self):
        return len(self._masks)

    def set_flux_bc(self, member, Q):
        self._check(self._lib.lbm_batch_set_flux_bc(self._h, int(member), float(Q)))

    def step(self, n=1):
        self._check(self._lib.lbm_batch_step(self._h, int(n)))

    def get_flux(self, member, face=LBM_FACE_ZMIN):
        q, r = C.c_double(), C.c_double()
        self._check(self._lib.lbm_batch_get_flux(self._h, int(member), face, C.byref(q), C.byref(r)))
        return q.value, r.value

    def distributions(self, member):
        f = np.empty((19,) + self._masks[member].shape)
        self._check(self._lib.lbm_batch_get_distributions(self._h, int(member), _ptr(f, C.c_double)))
        return f

    def set_distributions(self, member, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        if f.shape != (19,) + self._masks[member].shape:
            raise ValueError("f must have shape (19,) + mask.shape")
        self._check(self._lib.lbm_batch_set_distributions(self._h, int(member), _ptr(f, C.c_double)))

    def fields(self, member):
        shape = self._masks[member].shape
        arrs = [np.empty(shape) for _ in range(4)]
        self._check(self._lib.lbm_batch_get_fields(self._h, int(member), *[_ptr(a, C.c_double) for a in arrs]))
        return tuple(arrs)

    def info(self):
        v = [C.c_int64() for _ in range(3)]
        self._check(self._lib.lbm_batch_get_info(self._h, *[C.byref(x) for x in v]))
        return dict(zip(("n_pore", "n_tiles", "steps"), (x.value for x in v)))

    def time_step(self, n):
        ms = C.c_float()
        self._check(self._lib.lbm_batch_time_step(self._h, int(n), C.byref(ms)))
        return ms.value

    def set_config(self, config):
        """Launch configuration (LBM_BATCH_*): per-step launches under a graph,
        one persistent launch per call, or the AA pattern, each with a 64- or
        48-register cap."""
        self._check(self._lib.lbm_batch_set_config(self._h, int(config)))

    def autotune(self, trial_steps=200):
        """Time every configuration on this ensemble and keep the fastest; the
        state is left as it was.  Returns (best, ms per step of each)."""
        best = C.c_int()
        ms = (C.c_float * LBM_BATCH_NCONFIG)()
        self._check(self._lib.lbm_batch_autotune(self._h, int(trial_steps), C.byref(best), ms))
        return best.value, [float(v) for v in ms]

    def check_barrier(self, timeout_ms=20.0):
        """(completes, times_out) of the persistent launch's grid barrier."""
        a, b = C.c_int(), C.c_int()
        self._check(self._lib.lbm_batch_check_barrier(self._h, float(timeout_ms), C.byref(a), C.byref(b)))
        return bool(a.value), bool(b.value)


class WarmStartNet:
    """The warm-start network (lbm_wsnet_*): `levels` resolution levels with
    base * 2^l channels at level l (the specified network: 4 levels, 32 base
    channels); 4 output fields: u / u_D and the pressure gradient G."""

    N_OUT = 4

    def __init__(self, levels=4, base=32, stream=None):
        lib = load_library()
        h = _P()
        st = lib.lbm_wsnet_create(int(levels), int(base), C.byref(h))
        if st != LBM_OK:
            raise LBMError(st, "lbm_wsnet_create(%d, %d)" % (levels, base))
        self._h, self._lib, self.levels, self.base = h, lib, int(levels), int(base)
        n = C.c_int64()
        self._check(lib.lbm_wsnet_num_params(h, C.byref(n)))
        self.n_params = n.value
        if stream is not None:
            hs = getattr(stream, "cuda_stream", stream)
            self._check(lib.lbm_wsnet_set_stream(h, _P(hs) if hs else None))

    def _check(self, st):
        if st != LBM_OK:
            raise LBMError(st, self._lib.lbm_wsnet_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_wsnet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def layer_shapes(self):
        """(cout, cin) of the convolutions in the library's parameter order."""
        c = [self.base << l for l in range(self.levels)]
        shapes = [(c[0], 1), (c[0], c[0])]
        for l in range(1, self.levels):
            shapes += [(c[l], c[l - 1]), (c[l], c[l])]
        for l in range(self.levels - 2, -1, -1):
            shapes += [(c[l], c[l + 1]), (c[l], c[l])]
        return shapes + [(self.N_OUT, c[0])]

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        if p.size != self.n_params:
            raise ValueError("expected %d parameters" % self.n_params)
        self._check(self._lib.lbm_wsnet_set_params(self._h, _ptr(p, C.c_float)))

    def params(self):
        p = np.empty(self.n_params, np.float32)
        self._check(self._lib.lbm_wsnet_get_params(self._h, _ptr(p, C.c_float)))
        return p

    def loss_grad(self, masks, targets):
        masks = np.ascontiguousarray(masks, dtype=np.uint8)
        targets = np.ascontiguousarray(targets, dtype=np.float32)
        B, nz, ny, nx = masks.shape
        if targets.shape != (B, self.N_OUT, nz, ny, nx):
            raise ValueError("targets must have shape %s" % ((B, self.N_OUT, nz, ny, nx),))
        loss = C.c_double()
        g = np.empty(self.n_params, np.float32)
        self._check(self._lib.lbm_wsnet_loss_grad(self._h, _ptr(masks, C.c_uint8), _ptr(targets, C.c_float), B,
                                                  nx, ny, nz, C.byref(loss), _ptr(g, C.c_float)))
        return loss.value, g

    def train(self, masks, targets, epochs, batch, lr, seed=0):
        masks = np.ascontiguousarray(masks, dtype=np.uint8)
        targets = np.ascontiguousarray(targets, dtype=np.float32)
        S, nz, ny, nx = masks.shape
        if targets.shape != (S, self.N_OUT, nz, ny, nx):
            raise ValueError("targets must have shape %s" % ((S, self.N_OUT, nz, ny, nx),))
        rng = np.random.default_rng(seed)
        order = np.ascontiguousarray(np.concatenate([rng.permutation(S) for _ in range(epochs)]).astype(np.int32))
        hist = np.empty(epochs, np.float32)
        self._check(self._lib.lbm_wsnet_train(self._h, _ptr(masks, C.c_uint8), _ptr(targets, C.c_float), S, nx, ny,
                                              nz, int(epochs), int(batch), float(lr), _ptr(order, C.c_int),
                                              _ptr(hist, C.c_float)))
        return hist

    def predict(self, mask):
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        nz, ny, nx = mask.shape
        y = np.empty((self.N_OUT, nz, ny, nx), np.float32)
        self._check(self._lib.lbm_wsnet_predict(self._h, _ptr(mask, C.c_uint8), nx, ny, nz, _ptr(y, C.c_float)))
        return y

    def release_buffers(self):
        self._check(self._lib.lbm_wsnet_release_buffers(self._h))


def conv3d_bf16(op, inp, aux, w, bias, relu, out, batch, nx, ny, nz, cin, cout, stream=None, reps=None):
    """lbm_conv3d_bf16 on device pointers (ints, e.g. torch tensor.data_ptr());
    with reps, lbm_conv3d_bf16_time: returns the mean ms of one launch."""
    lib = load_library()
    hs = getattr(stream, "cuda_stream", stream) if stream is not None else None
    args = [int(op), _P(inp), _P(aux) if aux else None, _P(w), C.cast(_P(bias), _FP) if bias else None, int(relu),
            _P(out), int(batch), int(nx), int(ny), int(nz), int(cin), int(cout)]
    if reps is None:
        st = lib.lbm_conv3d_bf16(*args, _P(hs) if hs else None)
        ms = None
    else:
        t = C.c_float()
        st = lib.lbm_conv3d_bf16_time(*args, int(reps), C.byref(t), _P(hs) if hs else None)
        ms = t.value
    if st != LBM_OK:
        raise LBMError(st, "lbm_conv3d_bf16(op %d, cin %d, cout %d)" % (op, cin, cout))
    return ms


class ColorLattice:
    """Two-fluid colour model (lbm_color_*).  mask: uint8 [z][y][x], 1 = solid."""

    def __init__(self, mask, tau, alpha, beta=0.95, phi_s=-1.0, precision="fp64", stream=None):
        lib = load_library()
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        self.nz, self.ny, self.nx = mask.shape
        self.shape = mask.shape
        h = _P()
        st = lib.lbm_color_create(_ptr(mask, C.c_uint8), self.nx, self.ny, self.nz, float(tau), float(alpha),
                                  float(beta), float(phi_s), PRECISIONS[precision], C.byref(h))
        if st != LBM_OK:
            raise LBMError(st, lib.lbm_color_last_error(None).decode())
        self._h, self._lib = h, lib
        if stream is not None:
            hs = getattr(stream, "cuda_stream", stream)
            self._check(lib.lbm_color_set_stream(h, _P(hs) if hs else None))

    def _check(self, st):
        if st != LBM_OK:
            raise LBMError(st, self._lib.lbm_color_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_color_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_flux_bc(self, Q, phi_in=1.0):
        self._check(self._lib.lbm_color_set_flux_bc(self._h, float(Q), float(phi_in)))

    def set_phase(self, phi, rho=None):
        phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(self.shape)
        rho = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64).reshape(self.shape)
        self._check(self._lib.lbm_color_set_phase(self._h, _ptr(phi, C.c_double), _ptr(rho, C.c_double)))

    def set_state(self, f, A, B):
        cv = [np.ascontiguousarray(a, dtype=np.float64) for a in (f, A, B)]
        self._check(self._lib.lbm_color_set_state(self._h, *[_ptr(a, C.c_double) for a in cv]))

    def state(self):
        f = np.empty((19,) + self.shape)
        A = np.empty((7,) + self.shape)
        B = np.empty((7,) + self.shape)
        self._check(self._lib.lbm_color_get_state(self._h, *[_ptr(a, C.c_double) for a in (f, A, B)]))
        return f, A, B

    def step(self, n=1):
        self._check(self._lib.lbm_color_step(self._h, int(n)))

    def fields(self):
        arrs = [np.empty(self.shape) for _ in range(5)]
        self._check(self._lib.lbm_color_get_fields(self._h, *[_ptr(a, C.c_double) for a in arrs]))
        return tuple(arrs)

    def get_flux(self, face=LBM_FACE_ZMIN):
        q, r = C.c_double(), C.c_double()
        self._check(self._lib.lbm_color_get_flux(self._h, face, C.byref(q), C.byref(r)))
        return q.value, r.value
