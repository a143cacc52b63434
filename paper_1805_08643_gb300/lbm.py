"""ctypes binding of the C ABI in include/lbm.h (argument marshalling only).

Every numerical step runs in liblbm.so's CUDA kernels.  PyTorch provides the
device memory (``lbm_bind``) and the stream (the current torch stream).  If
the library is missing this module raises at import: there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# LBM_DEBUG_LIBRARY=1: the debug build (kernel index checks, _build.build(debug=True))
LIB_PATH = os.path.join(HERE, "liblbm_debug.so" if os.environ.get("LBM_DEBUG_LIBRARY") == "1" else "liblbm.so")

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NONFINITE, ERR_EOS_DOMAIN, ERR_TIMEOUT, ERR_STATE, ERR_BOUNDS = range(9)
OPERATORS = {"orth": 0, "nonorth": 1, "nonorth_d3q15": 2}
LATTICE_Q = {"orth": 19, "nonorth": 19, "nonorth_d3q15": 15}
PRECISIONS = {"f64": 0, "f32": 1, "f16": 2}
EOS_KINDS = {"cs": 0, "exp": 1, "none": 2}

# Every symbol include/lbm.h declares, with (restype, argtypes).
_c_int, _c_double, _vp = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_szp = ctypes.POINTER(ctypes.c_size_t)
_llp = ctypes.POINTER(ctypes.c_longlong)


class LbmEos(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("a", _c_double), ("b", _c_double), ("R", _c_double),
                ("T", _c_double), ("psi0", _c_double), ("rho0", _c_double)]


class LbmRates(ctypes.Structure):
    _fields_ = [("s_e", _c_double), ("s_nu", _c_double), ("s_q", _c_double), ("s_pi", _c_double),
                ("s_eps", _c_double), ("s_m", _c_double)]


SIGNATURES = {
    "lbm_create": (_c_int, [ctypes.POINTER(ctypes.c_int * 3), ctypes.POINTER(LbmEos), _c_double,
                            ctypes.POINTER(LbmRates), _c_int, _c_int, _c_double, _vp,
                            ctypes.POINTER(_vp)]),
    "lbm_buffer_bytes": (_c_int, [_vp, _szp, _szp, _szp]),
    "lbm_bind": (_c_int, [_vp, _vp, _vp, _vp, _vp]),
    "lbm_init_droplet": (_c_int, [_vp, _dp, _c_double, _c_double, _c_double, _c_double]),
    "lbm_init_droplets": (_c_int, [_vp, _c_int, _dp, _dp, _c_double, _c_double, _c_double]),
    "lbm_init_flat": (_c_int, [_vp, _c_int, _c_double, _c_double, _c_double, _c_double, _c_double]),
    "lbm_init_field": (_c_int, [_vp, _vp, _c_int, _c_double]),
    "lbm_step": (_c_int, [_vp, _c_int]),
    "lbm_moments": (_c_int, [_vp, _vp, _vp, _c_int]),
    "lbm_get_populations": (_c_int, [_vp, _vp, _c_int]),
    "lbm_set_populations": (_c_int, [_vp, _vp, _c_int]),
    "lbm_diag": (_c_int, [_vp, _dp]),
    "lbm_check": (_c_int, [_vp]),
    "lbm_set_check_interval": (_c_int, [_vp, _c_int]),
    "lbm_set_profiling": (_c_int, [_vp, _c_int]),
    "lbm_kernel_times": (_c_int, [_vp, _dp, _llp, _dp, _llp]),
    "lbm_set_tuning": (_c_int, [_vp, _c_int, _c_int, _c_int]),
    "lbm_set_eos_arith": (_c_int, [_vp, _c_int]),
    "lbm_set_wait_budget": (_c_int, [_vp, _c_int, _c_int]),
    "lbm_set_variable_viscosity": (_c_int, [_vp, _c_double, _c_double, _c_double, _c_double]),
    "lbm_get_tuning": (_c_int, [_vp, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int), ctypes.POINTER(_c_int)]),
    "lbm_step_count": (ctypes.c_longlong, [_vp]),
    "lbm_step_static": (_c_int, [_vp, _vp, _vp]),
    "lbm_batch_box_bytes": (ctypes.c_size_t, [_c_int, ctypes.POINTER(ctypes.c_int * 3)]),
    "lbm_batch_create": (_c_int, [_c_int, _c_int, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)]),
    "lbm_batch_add": (_c_int, [_vp, ctypes.POINTER(ctypes.c_int * 3), ctypes.POINTER(LbmEos), _c_double,
                               ctypes.POINTER(LbmRates), _c_int, _c_double, ctypes.POINTER(_c_int)]),
    "lbm_batch_remove": (_c_int, [_vp, _c_int]),
    "lbm_batch_init_droplet": (_c_int, [_vp, _c_int, _dp, _c_double, _c_double, _c_double, _c_double]),
    "lbm_batch_init_flat": (_c_int, [_vp, _c_int, _c_int, _c_double, _c_double, _c_double, _c_double, _c_double]),
    "lbm_batch_set_tuning": (_c_int, [_vp, _c_int, _c_int, _c_int]),
    "lbm_batch_step": (_c_int, [_vp, _c_int]),
    "lbm_batch_moments": (_c_int, [_vp, _c_int, _vp, _vp, _c_int]),
    "lbm_batch_diag": (_c_int, [_vp, _c_int, _dp]),
    "lbm_batch_max_du": (_c_int, [_vp, _c_int, ctypes.POINTER(_c_int), _dp]),
    "lbm_batch_check": (_c_int, [_vp]),
    "lbm_batch_info": (_c_int, [_vp, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int), _szp]),
    "lbm_batch_box_steps": (ctypes.c_longlong, [_vp, _c_int]),
    "lbm_batch_graph_builds": (ctypes.c_longlong, [_vp]),
    "lbm_batch_last_error": (ctypes.c_char_p, [_vp]),
    "lbm_batch_destroy": (None, [_vp]),
    "lbm_destroy": (None, [_vp]),
    "lbm_last_error": (ctypes.c_char_p, [_vp]),
    "lbm_status_string": (ctypes.c_char_p, [_c_int]),
}


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1805_08643_gb300._build.build() "
                          "(the CUDA path has no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = load_library()


class LBMError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        name = lib.lbm_status_string(status).decode()
        super().__init__(f"{where}: {name}" + (f" ({detail})" if detail else ""))


@dataclass
class Rates:
    """Relaxation rates (see lbm_rates in include/lbm.h)."""

    s_e: float = 1.1
    s_nu: float = 1.0
    s_q: float = 1.1
    s_pi: float = 1.1
    s_eps: float = 1.1
    s_m: float = 1.1


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Lattice:
    """One periodic box on the current CUDA device: D3Q19 with the orthogonal or
    non-orthogonal operator, or the D3Q15 non-orthogonal variant
    (``operator="nonorth_d3q15"``).

    Device buffers come from PyTorch and are bound to the C context; work runs
    on the current torch stream (or ``stream``, a torch.cuda.Stream).
    """

    def __init__(self, grid, operator="nonorth", precision="f64", eos="cs", a=1.0, b=4.0, R=1.0,
                 T=0.0, psi0=1.0, rho0=1.0, G=-1.0, rates: Rates | None = None, sigma=0.0,
                 stream=None, torch_buffers=True):
        import torch

        self.grid = tuple(int(v) for v in grid)
        self.n = self.grid[0] * self.grid[1] * self.grid[2]
        self.operator, self.precision = operator, precision
        self.q = LATTICE_Q[operator]
        rates = rates or Rates()
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        eos_s = LbmEos(EOS_KINDS[eos], a, b, R, T, psi0, rho0)
        rates_s = LbmRates(rates.s_e, rates.s_nu, rates.s_q, rates.s_pi, rates.s_eps, rates.s_m)
        g = (ctypes.c_int * 3)(*self.grid)
        handle = ctypes.c_void_p()
        st = lib.lbm_create(ctypes.byref(g), ctypes.byref(eos_s), G, ctypes.byref(rates_s),
                            OPERATORS[operator], PRECISIONS[precision], sigma,
                            ctypes.c_void_p(self._stream.cuda_stream), ctypes.byref(handle))
        if st != OK:
            raise LBMError(st, "lbm_create")
        self._h = handle
        self._buffers = []
        if torch_buffers:
            pb, sb, xb = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
            self._check(lib.lbm_buffer_bytes(self._h, ctypes.byref(pb), ctypes.byref(sb),
                                             ctypes.byref(xb)), "lbm_buffer_bytes")
            dev = torch.device("cuda", torch.cuda.current_device())
            self._buffers = [torch.empty(int(v), dtype=torch.uint8, device=dev)
                             for v in (pb.value, pb.value, sb.value, xb.value)]
            self._check(lib.lbm_bind(self._h, *[ctypes.c_void_p(t.data_ptr()) for t in self._buffers]),
                        "lbm_bind")

    # -------------------------------------------------------------- plumbing
    def _check(self, status, where):
        if status != OK:
            raise LBMError(status, where, lib.lbm_last_error(self._h).decode())

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib.lbm_destroy(self._h)
            self._h = None
            self._buffers = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -------------------------------------------------------------- state
    def init_droplet(self, centre, R, W, rho_l, rho_v):
        c = (ctypes.c_double * 3)(*centre)
        self._check(lib.lbm_init_droplet(self._h, c, R, W, rho_l, rho_v), "lbm_init_droplet")

    def init_droplets(self, centres, radii, W, rho_l, rho_v):
        c = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, 3)
        r = np.ascontiguousarray(radii, dtype=np.float64).reshape(-1)
        self._check(lib.lbm_init_droplets(self._h, len(r), c.ctypes.data_as(_dp), r.ctypes.data_as(_dp),
                                          W, rho_l, rho_v), "lbm_init_droplets")

    def init_flat(self, axis, lo, hi, W, rho_l, rho_v):
        self._check(lib.lbm_init_flat(self._h, axis, lo, hi, W, rho_l, rho_v), "lbm_init_flat")

    def init_field(self, rho, rho_ref):
        """rho: numpy array (host) or CUDA torch tensor of N float64, x fastest."""
        if isinstance(rho, np.ndarray):
            a = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
            assert a.size == self.n
            self._check(lib.lbm_init_field(self._h, _ptr(a), 0, rho_ref), "lbm_init_field")
        else:
            assert rho.is_cuda and rho.dtype.is_floating_point and rho.numel() == self.n
            t = rho.contiguous().double()
            self._check(lib.lbm_init_field(self._h, ctypes.c_void_p(t.data_ptr()), 1, rho_ref),
                        "lbm_init_field")

    def step(self, n=1):
        self._check(lib.lbm_step(self._h, int(n)), "lbm_step")

    @property
    def steps(self):
        return lib.lbm_step_count(self._h)

    def moments(self):
        """(rho, u) as float64 numpy arrays of shapes (Nz,Ny,Nx) and (3,Nz,Ny,Nx)."""
        nx, ny, nz = self.grid
        rho = np.empty(self.n)
        u = np.empty(3 * self.n)
        self._check(lib.lbm_moments(self._h, _ptr(rho), _ptr(u), 0), "lbm_moments")
        return rho.reshape(nz, ny, nx), u.reshape(3, nz, ny, nx)

    def moments_device(self, rho_t, u_t):
        """Write rho (N) and u (3N) into CUDA float64 tensors."""
        self._check(lib.lbm_moments(self._h, ctypes.c_void_p(rho_t.data_ptr()),
                                    ctypes.c_void_p(u_t.data_ptr()), 1), "lbm_moments")

    def populations(self):
        nx, ny, nz = self.grid
        f = np.empty(self.q * self.n)
        self._check(lib.lbm_get_populations(self._h, _ptr(f), 0), "lbm_get_populations")
        return f.reshape(self.q, nz, ny, nx)

    def set_populations(self, f):
        a = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        assert a.size == self.q * self.n
        self._check(lib.lbm_set_populations(self._h, _ptr(a), 0), "lbm_set_populations")

    def diag(self):
        out = (ctypes.c_double * 5)()
        self._check(lib.lbm_diag(self._h, out), "lbm_diag")
        return {"mass": out[0], "momentum": (out[1], out[2], out[3]), "max_u": out[4]}

    def check(self):
        return lib.lbm_check(self._h)

    def set_check_interval(self, k):
        self._check(lib.lbm_set_check_interval(self._h, int(k)), "lbm_set_check_interval")

    def set_tuning(self, single_pass=True, tile=1, z_planes=0):
        """single_pass: False / True (register-prefetch kernel) / "tma" (bulk-copy kernel) /
        "onchip" (psi evaluated on chip by producer warps; Nx even) / "lagged" (the next psi pass one plane
        behind the fused pass in one cooperative launch; Nx even) / "queue" (fused and next-psi tile jobs from
        an ordered work list in one cooperative launch; Nx even; the only single pass of a D3Q15 box and the
        default with FP32 storage)."""
        if isinstance(single_pass, str):
            modes = {"tma": 2, "onchip": 3, "lagged": 4, "queue": 5}
            if single_pass not in modes:
                raise ValueError(f"unknown single_pass mode {single_pass!r}")
            mode = modes[single_pass]
        else:
            mode = int(bool(single_pass))
        self._check(lib.lbm_set_tuning(self._h, mode, int(tile), int(z_planes)), "lbm_set_tuning")

    def set_wait_budget(self, spin_limit=0, inject_unreachable=False):
        """Polls before a device-side wait gives up (0: the default); inject_unreachable makes the cross-block
        waits of the "lagged" and "queue" modes wait for a count no block reaches (a test of the timeout path)."""
        self._check(lib.lbm_set_wait_budget(self._h, int(spin_limit), 1 if inject_unreachable else 0),
                    "lbm_set_wait_budget")

    def set_variable_viscosity(self, rho_l, rho_v, nu_l, nu_v):
        """nu linear in rho between (rho_v, nu_v) and (rho_l, nu_l), clamped; nu_l = nu_v = 0 switches it off."""
        self._check(lib.lbm_set_variable_viscosity(self._h, rho_l, rho_v, nu_l, nu_v), "lbm_set_variable_viscosity")

    def set_eos_arith(self, mode="f64"):
        """EOS radicand arithmetic of the psi pass: "f64" or "f32x2" (compensated FP32 pairs)."""
        self._check(lib.lbm_set_eos_arith(self._h, {"f64": 0, "f32x2": 1}[mode]), "lbm_set_eos_arith")

    def tuning(self):
        sp, t, z = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(lib.lbm_get_tuning(self._h, ctypes.byref(sp), ctypes.byref(t), ctypes.byref(z)), "lbm_get_tuning")
        return {"single_pass": {0: False, 1: True, 2: "tma", 3: "onchip", 4: "lagged", 5: "queue"}[sp.value],
                "tile": t.value,
                "z_planes": z.value}

    def set_profiling(self, on=True):
        self._check(lib.lbm_set_profiling(self._h, 1 if on else 0), "lbm_set_profiling")

    def kernel_times(self):
        mp, mf = ctypes.c_double(), ctypes.c_double()
        npsi, nf = ctypes.c_longlong(), ctypes.c_longlong()
        self._check(lib.lbm_kernel_times(self._h, ctypes.byref(mp), ctypes.byref(npsi), ctypes.byref(mf),
                                         ctypes.byref(nf)), "lbm_kernel_times")
        return {"psi_ms": mp.value, "psi_launches": npsi.value, "fused_ms": mf.value,
                "fused_launches": nf.value}


class Batch:
    """Many boxes advanced together (include/lbm.h, "batches"); FP32 arithmetic."""

    def __init__(self, precision="f32", eos="cs", hbm_budget_bytes=1 << 40, stream=None):
        import torch

        self.precision = precision
        self.eos = eos
        # graphs cannot be captured on the legacy default stream: a batch gets its own
        self._stream = stream if stream is not None else torch.cuda.Stream()
        h = ctypes.c_void_p()
        st = lib.lbm_batch_create(PRECISIONS[precision], EOS_KINDS[eos], int(hbm_budget_bytes),
                                  ctypes.c_void_p(self._stream.cuda_stream), ctypes.byref(h))
        if st != OK:
            raise LBMError(st, "lbm_batch_create")
        self._h = h
        self.grids = {}

    def _check(self, st, where):
        if st != OK:
            raise LBMError(st, where, lib.lbm_batch_last_error(self._h).decode())

    @property
    def stream(self):
        """The torch.cuda.Stream the batch's work runs on."""
        return self._stream

    @staticmethod
    def box_bytes(precision, grid):
        return lib.lbm_batch_box_bytes(PRECISIONS[precision], ctypes.byref((ctypes.c_int * 3)(*grid)))

    def add(self, grid, operator="nonorth", a=1.0, b=4.0, R=1.0, T=0.0, psi0=1.0, rho0=1.0, G=-1.0,
            rates: Rates | None = None, sigma=0.0):
        rates = rates or Rates()
        g = (ctypes.c_int * 3)(*grid)
        e = LbmEos(EOS_KINDS[self.eos], a, b, R, T, psi0, rho0)
        r = LbmRates(rates.s_e, rates.s_nu, rates.s_q, rates.s_pi, rates.s_eps, rates.s_m)
        i = ctypes.c_int()
        self._check(lib.lbm_batch_add(self._h, ctypes.byref(g), ctypes.byref(e), G, ctypes.byref(r),
                                      OPERATORS[operator], sigma, ctypes.byref(i)), "lbm_batch_add")
        self.grids[i.value] = tuple(grid)
        return i.value

    def try_add(self, *args, **kw):
        """add(), or None when the HBM budget has no room."""
        try:
            return self.add(*args, **kw)
        except LBMError as e:
            if e.status == ERR_OOM:
                return None
            raise

    def remove(self, box):
        self._check(lib.lbm_batch_remove(self._h, box), "lbm_batch_remove")
        self.grids.pop(box, None)

    def init_droplet(self, box, centre, R, W, rho_l, rho_v):
        c = (ctypes.c_double * 3)(*centre)
        self._check(lib.lbm_batch_init_droplet(self._h, box, c, R, W, rho_l, rho_v), "lbm_batch_init_droplet")

    def init_flat(self, box, axis, lo, hi, W, rho_l, rho_v):
        self._check(lib.lbm_batch_init_flat(self._h, box, axis, lo, hi, W, rho_l, rho_v), "lbm_batch_init_flat")

    def set_tuning(self, tile=1, box=-1, z_planes=0):
        self._check(lib.lbm_batch_set_tuning(self._h, tile, box, z_planes), "lbm_batch_set_tuning")

    def step(self, n=1):
        self._check(lib.lbm_batch_step(self._h, int(n)), "lbm_batch_step")

    def moments(self, box):
        nx, ny, nz = self.grids[box]
        n = nx * ny * nz
        rho, u = np.empty(n), np.empty(3 * n)
        self._check(lib.lbm_batch_moments(self._h, box, _ptr(rho), _ptr(u), 0), "lbm_batch_moments")
        return rho.reshape(nz, ny, nx), u.reshape(3, nz, ny, nx)

    def diag(self, box):
        out = (ctypes.c_double * 5)()
        self._check(lib.lbm_batch_diag(self._h, box, out), "lbm_batch_diag")
        return {"mass": out[0], "momentum": (out[1], out[2], out[3]), "max_u": out[4]}

    def max_du(self, boxes):
        ids = (ctypes.c_int * len(boxes))(*boxes)
        out = (ctypes.c_double * max(len(boxes), 1))()
        self._check(lib.lbm_batch_max_du(self._h, len(boxes), ids, out), "lbm_batch_max_du")
        return [out[k] for k in range(len(boxes))]

    def check(self):
        return lib.lbm_batch_check(self._h)

    def info(self):
        lb, wi, by = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        self._check(lib.lbm_batch_info(self._h, ctypes.byref(lb), ctypes.byref(wi), ctypes.byref(by)), "lbm_batch_info")
        return {"live_boxes": lb.value, "work_items": wi.value, "bytes_used": by.value,
                "graph_builds": lib.lbm_batch_graph_builds(self._h)}

    def box_steps(self, box):
        return lib.lbm_batch_box_steps(self._h, box)

    def close(self):
        if getattr(self, "_h", None):
            lib.lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
