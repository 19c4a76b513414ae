"""Python binding of the C ABI in ``include/ucp.h`` (``libucp.so``).

Argument marshalling only: every step of the TREE path runs in the CUDA
kernels of the library.  Arrays may be numpy arrays (host) or torch CUDA
tensors (device, used in the order of the context's stream).  If the library
has not been built the import of :func:`lib` raises: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libucp.so")

UCP_OK, UCP_EINVAL, UCP_ENOMEM, UCP_ECUDA, UCP_ENONFINITE, UCP_ETIMEOUT, UCP_ESTATE = (
    0, -1, -2, -3, -4, -5, -6)
UCP_FP64, UCP_FP32C = 0, 1
UCP_ION, UCP_ELECTRON = 0, 1
UCP_POT_PLUMMER, UCP_POT_KELBG = 0, 1
UCP_WALK_SHAPES = 10
# (threads per block, blocks per SM, leaf sources staged by bulk copies) of each
# FP32C walk launch shape
WALK_SHAPE_TABLE = ((128, 7, 0), (896, 1, 0), (128, 8, 0), (1024, 1, 0), (256, 4, 0), (512, 2, 0),
                    (128, 7, 1), (896, 1, 1), (128, 8, 1), (256, 4, 1))

EXPORTS = ("ucp_create", "ucp_destroy", "ucp_set_state", "ucp_get_state", "ucp_tree_build",
           "ucp_tree_force", "ucp_step", "ucp_energy", "ucp_stats", "ucp_get_cube",
           "ucp_get_sorted", "ucp_get_tree", "ucp_get_counts", "ucp_profile", "ucp_profile_read",
           "ucp_strerror", "ucp_last_error", "ucp_selftest_wait_timeout", "ucp_create_batch",
           "ucp_energy_clouds", "ucp_get_cubes", "ucp_grad_ke_electrons", "ucp_set_graphs",
           "ucp_autotune", "ucp_set_walk_shape", "ucp_measure_peaks", "ucp_accel_vjp")


class UcpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class ucp_params(C.Structure):
    _fields_ = [("n", C.c_int64), ("leaf_cap", C.c_int32), ("precision", C.c_int32),
                ("q", C.c_double * 2), ("m", C.c_double * 2), ("cuda_stream", C.c_void_p),
                ("potential", C.c_int32), ("reserved", C.c_int32), ("lambda_ei", C.c_double)]


_lib = None


def lib():
    """Load ``libucp.so`` (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, dbl = C.c_void_p, C.c_int, C.c_int64, C.c_double
        L.ucp_create.argtypes = [C.POINTER(vp), C.POINTER(ucp_params)]
        L.ucp_destroy.argtypes = [vp]
        L.ucp_destroy.restype = None
        L.ucp_set_state.argtypes = [vp, vp, vp, vp, i32]
        L.ucp_get_state.argtypes = [vp, vp, vp, i32]
        L.ucp_tree_build.argtypes = [vp]
        L.ucp_tree_force.argtypes = [vp, dbl, dbl, vp, vp, i32]
        L.ucp_step.argtypes = [vp, dbl, i32, i64, dbl, dbl]
        L.ucp_energy.argtypes = [vp, dbl, dbl, vp]
        L.ucp_stats.argtypes = [vp, vp, i32]
        L.ucp_get_cube.argtypes = [vp, vp]
        L.ucp_get_sorted.argtypes = [vp, vp, vp, i32]
        L.ucp_get_tree.argtypes = [vp, C.POINTER(i64), i64, vp, vp, vp]
        L.ucp_get_counts.argtypes = [vp, vp, vp, i32]
        L.ucp_profile.argtypes = [vp, i32]
        L.ucp_profile_read.argtypes = [vp, C.POINTER(dbl), C.POINTER(i64)]
        L.ucp_create_batch.argtypes = [C.POINTER(vp), C.POINTER(ucp_params), C.c_int32, vp]
        L.ucp_create_batch.restype = C.c_int
        L.ucp_energy_clouds.argtypes = [vp, dbl, dbl, vp]
        L.ucp_energy_clouds.restype = C.c_int
        L.ucp_get_cubes.argtypes = [vp, vp]
        L.ucp_get_cubes.restype = C.c_int
        L.ucp_grad_ke_electrons.argtypes = [vp, dbl, i32, i64, dbl, dbl, i64, C.POINTER(dbl), vp,
                                             vp, i32]
        L.ucp_grad_ke_electrons.restype = C.c_int
        L.ucp_autotune.argtypes = [vp, dbl, dbl, C.POINTER(i32), C.POINTER(C.c_float)]
        L.ucp_autotune.restype = C.c_int
        L.ucp_accel_vjp.argtypes = [vp, dbl, dbl, vp, vp, i32]
        L.ucp_accel_vjp.restype = C.c_int
        L.ucp_measure_peaks.argtypes = [C.POINTER(C.c_double), vp]
        L.ucp_measure_peaks.restype = C.c_int
        L.ucp_set_walk_shape.argtypes = [vp, i32]
        L.ucp_set_walk_shape.restype = C.c_int
        L.ucp_set_graphs.argtypes = [vp, i32]
        L.ucp_set_graphs.restype = C.c_int
        L.ucp_selftest_wait_timeout.argtypes = [vp]
        L.ucp_selftest_wait_timeout.restype = C.c_int
        L.ucp_strerror.argtypes = [i32]
        L.ucp_strerror.restype = C.c_char_p
        L.ucp_last_error.argtypes = [vp]
        L.ucp_last_error.restype = C.c_char_p
        for name in ("ucp_create", "ucp_set_state", "ucp_get_state", "ucp_tree_build",
                     "ucp_tree_force", "ucp_step", "ucp_energy", "ucp_stats", "ucp_get_cube",
                     "ucp_get_sorted", "ucp_get_tree", "ucp_get_counts", "ucp_profile",
                     "ucp_profile_read"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def measure_peaks(stream=None):
    """Measured arithmetic throughput of the current device:
    {"fp32_fma_tflops", "fp32x2_fma_tflops", "rsqrt_gops", "fp64_fma_tflops"}."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    out = (C.c_double * 4)()
    rc = lib().ucp_measure_peaks(out, stream)
    if rc:
        raise UcpError(rc, "ucp_measure_peaks")
    return {"fp32_fma_tflops": out[0], "fp32x2_fma_tflops": out[1], "rsqrt_gops": out[2],
            "fp64_fma_tflops": out[3]}


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype):
    """(pointer, on_device) of a numpy array or torch tensor of the given dtype."""
    if a is None:
        return None, 0
    if _is_torch(a):
        import torch
        tdt = {np.float64: torch.float64, np.int8: torch.int8, np.int32: torch.int32,
               np.uint64: torch.uint64, np.uint32: torch.uint32}[dtype]
        if a.dtype != tdt or not a.is_contiguous():
            raise TypeError(f"tensor must be contiguous {tdt}")
        return a.data_ptr(), 1 if a.is_cuda else 0
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous:
        raise TypeError(f"array must be a C-contiguous numpy {np.dtype(dtype)}")
    return a.ctypes.data, 0


class Context:
    """One particle set on the current CUDA device (``ucp_create`` .. ``ucp_destroy``)."""

    def __init__(self, n, q=(1.0, -1.0), m=(1000.0, 1.0), leaf_cap=32, precision=UCP_FP64,
                 stream=None, kelbg_lambda=None, sizes=None):
        """``sizes``: particle counts of an ensemble of independent clouds
        (``ucp_create_batch``); their total must equal ``n``."""
        L = lib()
        p = ucp_params()
        p.n = int(n)
        p.leaf_cap = int(leaf_cap)
        p.precision = int(precision)
        p.q[0], p.q[1] = float(q[0]), float(q[1])
        p.m[0], p.m[1] = float(m[0]), float(m[1])
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except ImportError:
                stream = None
        p.cuda_stream = stream
        if kelbg_lambda is not None:
            p.potential = UCP_POT_KELBG
            p.lambda_ei = float(kelbg_lambda)
        self.n = int(n)
        self._h = C.c_void_p()
        if sizes is None:
            self.n_clouds = 1
            rc = L.ucp_create(C.byref(self._h), C.byref(p))
        else:
            sz = np.ascontiguousarray(sizes, dtype=np.int64)
            self.n_clouds = int(sz.shape[0])
            rc = L.ucp_create_batch(C.byref(self._h), C.byref(p), self.n_clouds, sz.ctypes.data)
        if rc:
            raise UcpError(rc, "ucp_create: " + L.ucp_strerror(rc).decode())

    def _check(self, rc, what):
        if rc:
            msg = lib().ucp_last_error(self._h).decode()
            raise UcpError(rc, f"{what}: {lib().ucp_strerror(rc).decode()}: {msg}")

    def close(self):
        if getattr(self, "_h", None):
            lib().ucp_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- state
    def set_state(self, pos, vel, species):
        pp, d1 = _ptr(pos, np.float64)
        vp, d2 = _ptr(vel, np.float64)
        sp, d3 = _ptr(species, np.int8)
        if not (d1 == d2 == d3):
            raise TypeError("pos, vel and species must all be host or all device arrays")
        self._check(lib().ucp_set_state(self._h, pp, vp, sp, d1), "ucp_set_state")

    def get_state(self, pos=None, vel=None):
        if pos is None and vel is None:
            pos = np.empty((self.n, 3))
            vel = np.empty((self.n, 3))
        pp, d1 = _ptr(pos, np.float64)
        vp, d2 = _ptr(vel, np.float64)
        self._check(lib().ucp_get_state(self._h, pp, vp, max(d1, d2)), "ucp_get_state")
        return pos, vel

    # -- the hot path
    def tree_build(self):
        self._check(lib().ucp_tree_build(self._h), "ucp_tree_build")

    def tree_force(self, theta, eps, acc=None, phi=None, want=True):
        """Accelerations (N, 3) and potentials (N,) in caller order; host
        arrays are allocated when none are given and ``want`` is true."""
        if acc is None and phi is None and want:
            acc = np.empty((self.n, 3))
            phi = np.empty(self.n)
        ap, d1 = _ptr(acc, np.float64)
        pp, d2 = _ptr(phi, np.float64)
        self._check(lib().ucp_tree_force(self._h, float(theta), float(eps), ap, pp, max(d1, d2)),
                    "ucp_tree_force")
        return acc, phi

    def step(self, dt_e, ion_substep_ratio, n_electron_steps, theta, eps):
        self._check(lib().ucp_step(self._h, float(dt_e), int(ion_substep_ratio),
                                   int(n_electron_steps), float(theta), float(eps)), "ucp_step")

    def energy(self, theta, eps):
        out = np.zeros(6)
        self._check(lib().ucp_energy(self._h, float(theta), float(eps), out.ctypes.data),
                    "ucp_energy")
        return out

    def accel_vjp(self, theta, eps, lam, mu=None):
        """mu = (d a / d x)^T lam at the current positions, tree held fixed
        (``ucp_accel_vjp``); lam and mu are N x 3 in caller order (numpy or
        torch CUDA tensors)."""
        if mu is None:
            mu = (np.zeros((self.n, 3)) if not _is_torch(lam)
                  else lam.new_zeros((self.n, 3)))
        lp, ld = _ptr(lam, np.float64)
        mp, md = _ptr(mu, np.float64)
        if ld != md:
            raise TypeError("lam and mu must both be host or both be device arrays")
        self._check(lib().ucp_accel_vjp(self._h, float(theta), float(eps), lp, mp, ld),
                    "ucp_accel_vjp")
        return mu

    def grad_ke_electrons(self, dt_e, ion_substep_ratio, n_steps, theta, eps,
                          checkpoint_every=None, grad_x=None, grad_v=None):
        """(L, dL/dx0, dL/dv0) for L = electron kinetic energy after ``n_steps``
        electron substeps from the current state (``ucp_grad_ke_electrons``)."""
        if checkpoint_every is None:
            checkpoint_every = n_steps
        if grad_x is None and grad_v is None:
            grad_x = np.empty((self.n, 3))
            grad_v = np.empty((self.n, 3))
        gx, d1 = _ptr(grad_x, np.float64)
        gv, d2 = _ptr(grad_v, np.float64)
        loss = C.c_double(0.0)
        self._check(lib().ucp_grad_ke_electrons(self._h, float(dt_e), int(ion_substep_ratio),
                                                int(n_steps), float(theta), float(eps),
                                                int(checkpoint_every), C.byref(loss), gx, gv,
                                                max(d1, d2)), "ucp_grad_ke_electrons")
        return loss.value, grad_x, grad_v

    def energy_clouds(self, theta, eps):
        out = np.zeros((self.n_clouds, 6))
        self._check(lib().ucp_energy_clouds(self._h, float(theta), float(eps), out.ctypes.data),
                    "ucp_energy_clouds")
        return out

    def get_cubes(self):
        out = np.zeros((self.n_clouds, 4))
        self._check(lib().ucp_get_cubes(self._h, out.ctypes.data), "ucp_get_cubes")
        return out

    def stats(self, reset=False):
        out = np.zeros(8, dtype=np.int64)
        self._check(lib().ucp_stats(self._h, out.ctypes.data, int(reset)), "ucp_stats")
        return out

    # -- inspection
    def get_cube(self):
        out = np.zeros(4)
        self._check(lib().ucp_get_cube(self._h, out.ctypes.data), "ucp_get_cube")
        return out

    def get_sorted(self):
        keys = np.zeros(self.n, dtype=np.uint64)
        ids = np.zeros(self.n, dtype=np.uint32)
        self._check(lib().ucp_get_sorted(self._h, keys.ctypes.data, ids.ctypes.data, 0),
                    "ucp_get_sorted")
        return keys, ids

    def get_tree(self):
        nn = C.c_int64(0)
        self._check(lib().ucp_get_tree(self._h, C.byref(nn), 0, None, None, None), "ucp_get_tree")
        k = nn.value
        topo = np.zeros((k, 4), dtype=np.int32)
        leaf = np.zeros(k, dtype=np.int8)
        geom = np.zeros((k, 20))
        self._check(lib().ucp_get_tree(self._h, C.byref(nn), k, topo.ctypes.data,
                                       leaf.ctypes.data, geom.ctypes.data), "ucp_get_tree")
        return {"begin": topo[:, 0], "end": topo[:, 1], "next": topo[:, 2], "depth": topo[:, 3],
                "is_leaf": leaf.astype(bool), "centre": geom[:, 0:3], "side": geom[:, 3],
                "S0": geom[:, 4], "M": geom[:, 5], "c": geom[:, 6:9], "D": geom[:, 9:12],
                "Q": geom[:, 12:18], "delta": geom[:, 18]}

    def get_counts(self):
        p2p = np.zeros(self.n, dtype=np.int32)
        m2p = np.zeros(self.n, dtype=np.int32)
        self._check(lib().ucp_get_counts(self._h, p2p.ctypes.data, m2p.ctypes.data, 0),
                    "ucp_get_counts")
        return p2p, m2p

    def selftest_wait_timeout(self):
        """Run the bounded-wait self-test; returns the status code (UCP_ETIMEOUT
        means the wait gave up and reported it as it should)."""
        return int(lib().ucp_selftest_wait_timeout(self._h))

    def autotune(self, theta, eps):
        """Pick the fastest launch shape of the FP32C walk on the current state;
        returns (shape index, ms for the walks of one 10-substep block)."""
        sh = C.c_int(0)
        ms = C.c_float(0.0)
        self._check(lib().ucp_autotune(self._h, float(theta), float(eps), C.byref(sh),
                                       C.byref(ms)), "ucp_autotune")
        return sh.value, ms.value

    def set_walk_shape(self, shape):
        """Set the FP32C walk launch shape (0 .. WALK_SHAPES-1) directly."""
        self._check(lib().ucp_set_walk_shape(self._h, int(shape)), "ucp_set_walk_shape")

    def set_graphs(self, enable=True):
        self._check(lib().ucp_set_graphs(self._h, int(bool(enable))), "ucp_set_graphs")

    def profile(self, enable=True):
        self._check(lib().ucp_profile(self._h, int(bool(enable))), "ucp_profile")

    def profile_read(self):
        ms = C.c_double(0.0)
        n = C.c_int64(0)
        self._check(lib().ucp_profile_read(self._h, C.byref(ms), C.byref(n)), "ucp_profile_read")
        return ms.value, n.value
