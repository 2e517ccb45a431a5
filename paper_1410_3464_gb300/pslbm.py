"""Thin ctypes binding of the C ABI in include/pslbm.h (argument marshalling
only: every step of the method runs in the CUDA library).

The library is loaded from paper_1410_3464_gb300/_lib/libpslbm.so; if it is
missing the binding raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpslbm.so")

MAX_SPECIES = 4
FP64, FP32, FP32_SOLUTE_F16, FP32_SOLUTE_BF16 = 0, 1, 2, 3
LIQUID, GAS, SOLID_D, SOLID_F, WALL, INLET, OUTLET = range(7)
F_RHO1, F_RHO2, F_UX, F_UY, F_CONC, F_TYPE, F_VOL, F_BUDGET = (1 << i for i in range(8))

STATUS = {0: "OK", -1: "ERR_PARAM", -2: "ERR_OOM", -3: "ERR_CUDA", -4: "ERR_NONFINITE",
          -5: "ERR_EOS_DOMAIN", -6: "ERR_TIMEOUT", -7: "ERR_STATE", -8: "ERR_NODEVICE"}

EXPORTS = ["pslbm_get_stream", "pslbm_set_stream", "pslbm_create", "pslbm_step", "pslbm_sync",
           "pslbm_profile_step",
           "pslbm_read_fields", "pslbm_info", "pslbm_device_bytes", "pslbm_destroy", "pslbm_last_error",
           "pslbm_batch_create", "pslbm_batch_step", "pslbm_batch_sync", "pslbm_batch_destroy",
           "pslbm_budget_device_noalloc", "pslbm_set_step_limit", "pslbm_estimate_device_bytes",
           "pslbm_server_create", "pslbm_server_submit", "pslbm_server_advance", "pslbm_server_poll",
           "pslbm_server_fetch", "pslbm_server_release", "pslbm_server_last_error", "pslbm_server_destroy",
           "pslbm_set_tile_shape", "pslbm_get_tile_shape", "pslbm_batch_get_tile_shape",
           "pslbm_set_staging", "pslbm_get_staging", "pslbm_batch_set_staging", "pslbm_batch_get_staging",
           "pslbm_monitor", "pslbm_batch_profile_step", "pslbm_batch_monitor"]

_D2 = C.c_double * 2
_DS = C.c_double * MAX_SPECIES


class Params(C.Structure):
    """Mirror of pslbm_params (field order and types as in include/pslbm.h)."""
    _fields_ = [
        ("struct_size", C.c_uint32), ("nx", C.c_int32), ("ny", C.c_int32),
        ("periodic_x", C.c_int32), ("periodic_y", C.c_int32), ("precision", C.c_int32),
        ("tau", _D2), ("G11", C.c_double), ("G12", C.c_double), ("G21", C.c_double),
        ("a0", C.c_double), ("rho10", C.c_double), ("rho20", C.c_double), ("w_adh", _D2),
        ("eos_a", C.c_double), ("eos_b", C.c_double), ("eos_R", C.c_double), ("eos_T", C.c_double),
        ("body_force", _D2), ("rho_ref", _D2),
        ("n_species", C.c_int32), ("idx_A", C.c_int32), ("idx_B", C.c_int32), ("idx_E", C.c_int32),
        ("idx_F", C.c_int32),
        ("J0", _DS), ("tau_g", _DS), ("conc_ref", _DS),
        ("k1", C.c_double), ("inv_Keq", C.c_double), ("k3", C.c_double),
        ("k2", C.c_double), ("k4", C.c_double), ("C_F_sat", C.c_double),
        ("gas_yield", C.c_double), ("inv_M_C", C.c_double), ("c_total_per_rho1", C.c_double),
        ("Vbar_D", C.c_double), ("Vbar_F", C.c_double), ("V_split", C.c_double), ("seed", C.c_uint64),
        ("rho_in_liq", _D2), ("rho_in_gas", _D2), ("rho_out", _D2), ("rho_out_gas", _D2),
        ("inlet_period_liq", C.c_int32), ("inlet_period_gas", C.c_int32), ("inlet_ramp", C.c_int32),
        ("conc_in", _DS), ("r1_surface_factor", C.c_double), ("rho_ref_gas", _D2),
        ("inlet_axis", C.c_int32), ("outlet_axis", C.c_int32), ("conc_scale", _DS),
    ]


def params_from_dict(d, precision=FP64):
    """Fill a Params block from a parameter dictionary (missing keys stay 0)."""
    p = Params()
    p.struct_size = C.sizeof(Params)
    p.precision = int(d.get("precision", precision))
    for name, ctype in Params._fields_:
        if name in ("struct_size", "precision") or name not in d:
            continue
        v = d[name]
        if issubclass(ctype, C.Array):
            arr = getattr(p, name)
            vals = list(v)
            for i in range(len(arr)):
                arr[i] = float(vals[i]) if i < len(vals) else 0.0
        elif ctype in (C.c_int32, C.c_uint32, C.c_uint64):
            setattr(p, name, int(v))
        else:
            setattr(p, name, float(v))
    return p


class ServerConfig(C.Structure):
    """Mirror of pslbm_server_config."""
    _fields_ = [("struct_size", C.c_uint32), ("precision", C.c_int32), ("hbm_budget_bytes", C.c_uint64),
                ("chunk_steps", C.c_int32), ("max_active", C.c_int32)]


REQ_QUEUED, REQ_ACTIVE, REQ_DONE, REQ_FAILED = 0, 1, 2, 3


class PslbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64, u32 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32
    lib.pslbm_get_stream.restype = vp
    lib.pslbm_set_stream.argtypes = [vp]
    lib.pslbm_create.argtypes = [vp, vp, vp, vp, vp, C.POINTER(Params), C.POINTER(vp)]
    lib.pslbm_step.argtypes = [vp, i64]
    lib.pslbm_sync.argtypes = [vp]
    lib.pslbm_profile_step.argtypes = [vp, i64, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.pslbm_read_fields.argtypes = [vp, u32, C.POINTER(vp)]
    lib.pslbm_info.argtypes = [vp, C.POINTER(i64), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
    lib.pslbm_device_bytes.argtypes = [vp, C.POINTER(C.c_uint64)]
    lib.pslbm_destroy.argtypes = [vp]
    lib.pslbm_last_error.argtypes = [vp]
    lib.pslbm_last_error.restype = C.c_char_p
    lib.pslbm_batch_create.argtypes = [i32, C.POINTER(vp), i32, i32, C.POINTER(vp)]
    lib.pslbm_batch_step.argtypes = [vp, i64]
    lib.pslbm_batch_sync.argtypes = [vp]
    lib.pslbm_batch_destroy.argtypes = [vp]
    lib.pslbm_budget_device_noalloc.argtypes = [vp, vp]
    lib.pslbm_set_step_limit.argtypes = [vp, i64]
    lib.pslbm_estimate_device_bytes.argtypes = [C.POINTER(Params), C.POINTER(C.c_uint64)]
    lib.pslbm_server_create.argtypes = [C.POINTER(ServerConfig), C.POINTER(vp)]
    lib.pslbm_server_submit.argtypes = [vp, vp, vp, vp, vp, vp, C.POINTER(Params), i64, C.c_double, i32,
                                        C.POINTER(C.c_uint64)]
    lib.pslbm_server_advance.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
    lib.pslbm_server_poll.argtypes = [vp, C.c_uint64, C.POINTER(i32), C.POINTER(i64), vp]
    lib.pslbm_server_fetch.argtypes = [vp, C.c_uint64, u32, C.POINTER(vp)]
    lib.pslbm_server_release.argtypes = [vp, C.c_uint64]
    lib.pslbm_server_last_error.argtypes = [vp]
    lib.pslbm_server_last_error.restype = C.c_char_p
    lib.pslbm_server_destroy.argtypes = [vp]
    lib.pslbm_set_tile_shape.argtypes = [vp, i32, i32]
    lib.pslbm_get_tile_shape.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
    lib.pslbm_batch_get_tile_shape.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
    lib.pslbm_set_staging.argtypes = [vp, i32]
    lib.pslbm_monitor.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_double), C.POINTER(C.c_uint32)]
    lib.pslbm_get_staging.argtypes = [vp, C.POINTER(i32), C.POINTER(i32)]
    lib.pslbm_batch_set_staging.argtypes = [vp, i32]
    lib.pslbm_batch_get_staging.argtypes = [vp, C.POINTER(i32), C.POINTER(i32)]
    lib.pslbm_batch_profile_step.argtypes = [vp, i64, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.pslbm_batch_monitor.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_uint32)]
    for name in EXPORTS:
        fn = getattr(lib, name)
        if name not in ("pslbm_get_stream", "pslbm_last_error", "pslbm_server_last_error"):
            fn.restype = C.c_int
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(st, h=None):
    if st != 0:
        msg = load().pslbm_last_error(h).decode(errors="replace")
        raise PslbmError(st, msg)


def get_stream():
    return load().pslbm_get_stream()


def set_stream(stream_ptr):
    _check(load().pslbm_set_stream(stream_ptr))


class Simulation:
    """One simulation handle (pslbm_create ... pslbm_destroy)."""

    def __init__(self, mask, params, rho1, rho2, conc=None, vol=None, precision=None):
        lib = load()
        d = dict(params)
        if precision is not None:
            d["precision"] = precision
        self.params = params_from_dict(d)
        self.nx, self.ny, self.ns = self.params.nx, self.params.ny, self.params.n_species
        shape = (self.ny, self.nx)
        self._mask = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8).reshape(shape))
        self._r1 = np.ascontiguousarray(np.asarray(rho1, dtype=np.float64).reshape(shape))
        self._r2 = np.ascontiguousarray(np.asarray(rho2, dtype=np.float64).reshape(shape))
        self._c = None if conc is None or self.ns == 0 else np.ascontiguousarray(
            np.asarray(conc, dtype=np.float64).reshape((self.ns,) + shape))
        self._v = None if vol is None else np.ascontiguousarray(np.asarray(vol, dtype=np.float64).reshape((2,) + shape))
        h = C.c_void_p()
        st = lib.pslbm_create(_ptr(self._mask), _ptr(self._r1), _ptr(self._r2), _ptr(self._c), _ptr(self._v),
                              C.byref(self.params), C.byref(h))
        _check(st)
        self.h = h

    def step(self, n=1):
        _check(load().pslbm_step(self.h, int(n)), self.h)

    def sync(self):
        _check(load().pslbm_sync(self.h), self.h)

    def profile_step(self, n=1):
        """Run n steps with per-kernel CUDA-event timing; returns
        ({'bulk', 'vop', 'amend'} mean ms per step, mean total ms per step)."""
        k = (C.c_double * 3)()
        t = C.c_double()
        _check(load().pslbm_profile_step(self.h, int(n), k, C.byref(t)), self.h)
        return dict(bulk=k[0], vop=k[1], amend=k[2]), t.value

    def set_tile_shape(self, tx, ty):
        _check(load().pslbm_set_tile_shape(self.h, int(tx), int(ty)), self.h)

    def tile_shape(self):
        tx, ty, tu = C.c_int32(), C.c_int32(), C.c_int32()
        _check(load().pslbm_get_tile_shape(self.h, C.byref(tx), C.byref(ty), C.byref(tu)), self.h)
        return tx.value, ty.value, bool(tu.value)

    def set_staging(self, mode):
        """-1: choose by timing, 0: plain-load bulk kernel, 1: TMA-staged,
        2: TMA-staged with one stage (three blocks per SM)."""
        _check(load().pslbm_set_staging(self.h, int(mode)), self.h)

    def staging(self):
        """(staging in use 0/1/2, staged kernels available)."""
        sg, av = C.c_int32(), C.c_int32()
        _check(load().pslbm_get_staging(self.h, C.byref(sg), C.byref(av)), self.h)
        return sg.value, bool(av.value)

    def monitor(self):
        """(steps taken, maximum rho_1 found by the last step, status bits):
        a 64-byte read, no kernel."""
        n, m, st = C.c_int64(), C.c_double(), C.c_uint32()
        _check(load().pslbm_monitor(self.h, C.byref(n), C.byref(m), C.byref(st)), self.h)
        return n.value, m.value, st.value

    def set_step_limit(self, limit):
        _check(load().pslbm_set_step_limit(self.h, int(limit)), self.h)

    def steps(self):
        t = C.c_int64()
        _check(load().pslbm_info(self.h, C.byref(t), None, None, None), self.h)
        return int(t.value)

    def device_bytes(self):
        b = C.c_uint64()
        _check(load().pslbm_device_bytes(self.h, C.byref(b)), self.h)
        return int(b.value)

    def read(self, fields=F_RHO1 | F_RHO2 | F_UX | F_UY | F_CONC | F_TYPE | F_VOL | F_BUDGET):
        """Read the selected fields into new numpy arrays (dict by name)."""
        N = self.nx * self.ny
        shape = (self.ny, self.nx)
        spec = [(F_RHO1, "rho1", np.float64, shape), (F_RHO2, "rho2", np.float64, shape),
                (F_UX, "ux", np.float64, shape), (F_UY, "uy", np.float64, shape),
                (F_CONC, "conc", np.float64, (self.ns,) + shape), (F_TYPE, "type", np.uint8, shape),
                (F_VOL, "vol", np.float64, (2,) + shape), (F_BUDGET, "budget", np.float64, (6 + self.ns,))]
        out = {}
        ptrs = []
        for bit, name, dt, shp in spec:
            if fields & bit:
                a = np.zeros(max(1, int(np.prod(shp))), dtype=dt)
                out[name] = a
                ptrs.append(a.ctypes.data_as(C.c_void_p))
        arr = (C.c_void_p * max(1, len(ptrs)))(*ptrs)
        _check(load().pslbm_read_fields(self.h, int(fields), arr), self.h)
        res = {}
        for bit, name, dt, shp in spec:
            if fields & bit:
                res[name] = out[name][: int(np.prod(shp))].reshape(shp)
        if "vol" in res:
            res["vol_d"], res["vol_f"] = res["vol"][0], res["vol"][1]
        del N
        return res

    def budget_device_noalloc(self, out_device_ptr):
        """Write the budget (6 + n_species doubles) to a caller-owned device
        buffer without allocating anything (see include/pslbm.h)."""
        _check(load().pslbm_budget_device_noalloc(self.h, out_device_ptr), self.h)

    def close(self):
        if getattr(self, "h", None):
            load().pslbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Several simulations stepped together over one packed tile list."""

    def __init__(self, sims, tile_x=0, tile_y=0):
        lib = load()
        self.sims = list(sims)
        arr = (C.c_void_p * len(self.sims))(*[s.h for s in self.sims])
        b = C.c_void_p()
        _check(lib.pslbm_batch_create(len(self.sims), arr, int(tile_x), int(tile_y), C.byref(b)))
        self.b = b

    def step(self, n=1):
        _check(load().pslbm_batch_step(self.b, int(n)))

    def sync(self):
        _check(load().pslbm_batch_sync(self.b))

    def tile_shape(self):
        tx, ty, tu = C.c_int32(), C.c_int32(), C.c_int32()
        _check(load().pslbm_batch_get_tile_shape(self.b, C.byref(tx), C.byref(ty), C.byref(tu)))
        return tx.value, ty.value, bool(tu.value)

    def set_staging(self, mode):
        _check(load().pslbm_batch_set_staging(self.b, int(mode)))

    def staging(self):
        sg, av = C.c_int32(), C.c_int32()
        _check(load().pslbm_batch_get_staging(self.b, C.byref(sg), C.byref(av)))
        return sg.value, bool(av.value)

    def profile_step(self, n=1):
        """Run n steps with per-kernel CUDA-event timing; returns
        ({'bulk', 'vop', 'amend'} mean ms per step, mean total ms per step)."""
        k = (C.c_double * 3)()
        t = C.c_double()
        _check(load().pslbm_batch_profile_step(self.b, int(n), k, C.byref(t)))
        return dict(bulk=k[0], vop=k[1], amend=k[2]), t.value

    def monitor(self):
        """(smallest step count over the members, OR of their status bits)."""
        n, st = C.c_int64(), C.c_uint32()
        _check(load().pslbm_batch_monitor(self.b, C.byref(n), C.byref(st)))
        return n.value, st.value

    def close(self):
        if getattr(self, "b", None):
            load().pslbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def estimate_device_bytes(params, precision=None):
    d = dict(params)
    if precision is not None:
        d["precision"] = precision
    prm = params_from_dict(d)
    b = C.c_uint64()
    _check(load().pslbm_estimate_device_bytes(C.byref(prm), C.byref(b)))
    return int(b.value)


class Server:
    """Continuous-batching request server (pslbm_server_*)."""

    def __init__(self, precision=FP32, hbm_budget_bytes=150 * 10**9, chunk_steps=200, max_active=1024):
        lib = load()
        cfg = ServerConfig()
        cfg.struct_size = C.sizeof(ServerConfig)
        cfg.precision = int(precision)
        cfg.hbm_budget_bytes = int(hbm_budget_bytes)
        cfg.chunk_steps = int(chunk_steps)
        cfg.max_active = int(max_active)
        s = C.c_void_p()
        st = lib.pslbm_server_create(C.byref(cfg), C.byref(s))
        if st != 0:
            raise PslbmError(st, "server create failed")
        self.s = s
        self._ns = {}

    def _check(self, st):
        if st != 0:
            raise PslbmError(st, load().pslbm_server_last_error(self.s).decode(errors="replace"))

    def submit(self, mask, params, rho1, rho2, conc=None, vol=None, step_budget=1000, stop_dv=0.0,
               keep_fields=False):
        prm = params_from_dict(dict(params))
        shape = (prm.ny, prm.nx)
        m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8).reshape(shape))
        r1 = np.ascontiguousarray(np.asarray(rho1, dtype=np.float64).reshape(shape))
        r2 = np.ascontiguousarray(np.asarray(rho2, dtype=np.float64).reshape(shape))
        c = None if conc is None or prm.n_species == 0 else np.ascontiguousarray(
            np.asarray(conc, dtype=np.float64).reshape((prm.n_species,) + shape))
        v = None if vol is None else np.ascontiguousarray(np.asarray(vol, dtype=np.float64).reshape((2,) + shape))
        rid = C.c_uint64()
        self._check(load().pslbm_server_submit(self.s, _ptr(m), _ptr(r1), _ptr(r2), _ptr(c), _ptr(v), C.byref(prm),
                                               int(step_budget), float(stop_dv), int(bool(keep_fields)),
                                               C.byref(rid)))
        self._ns[rid.value] = (prm.n_species, prm.nx, prm.ny)
        return rid.value

    def advance(self):
        a, q, d = C.c_int32(), C.c_int32(), C.c_int32()
        self._check(load().pslbm_server_advance(self.s, C.byref(a), C.byref(q), C.byref(d)))
        return a.value, q.value, d.value

    def poll(self, rid):
        ns = self._ns[rid][0]
        st, n = C.c_int32(), C.c_int64()
        b = np.zeros(6 + ns)
        self._check(load().pslbm_server_poll(self.s, int(rid), C.byref(st), C.byref(n), b.ctypes.data_as(C.c_void_p)))
        return st.value, n.value, (b if st.value == REQ_DONE else None)

    def fetch(self, rid):
        ns, nx, ny = self._ns[rid]
        shape = (ny, nx)
        spec = [(F_RHO1, "rho1", np.float64, shape), (F_RHO2, "rho2", np.float64, shape),
                (F_UX, "ux", np.float64, shape), (F_UY, "uy", np.float64, shape),
                (F_CONC, "conc", np.float64, (ns,) + shape), (F_TYPE, "type", np.uint8, shape),
                (F_VOL, "vol", np.float64, (2,) + shape)]
        if ns == 0:
            spec = [s for s in spec if s[0] != F_CONC]
        bits, outs, ptrs = 0, {}, []
        for bit, name, dt, shp in spec:
            a = np.zeros(shp, dtype=dt)
            outs[name] = a
            ptrs.append(a.ctypes.data_as(C.c_void_p))
            bits |= bit
        arr = (C.c_void_p * len(ptrs))(*ptrs)
        self._check(load().pslbm_server_fetch(self.s, int(rid), bits, arr))
        return outs

    def release(self, rid):
        self._check(load().pslbm_server_release(self.s, int(rid)))

    def close(self):
        if getattr(self, "s", None):
            load().pslbm_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
