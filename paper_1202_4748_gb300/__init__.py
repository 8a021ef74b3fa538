"""Python binding of liblbfluct: GB300 fluctuating non-ideal-fluid lattice Boltzmann.

A thin ctypes layer over the C ABI of ``include/lbfluct.h`` (same entry-point
names, argument marshalling only).  Every step of the method runs in the CUDA
kernels of the shared library; PyTorch is used only to allocate the device
workspace and to obtain the current CUDA stream.  Importing this package
fails loudly if the library has not been built (``__graft_entry__.build()``
or ``python -m paper_1202_4748_gb300._build``).
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbfluct.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("liblbfluct.so is not built (expected at %s); build it with "
                      "`python -m paper_1202_4748_gb300._build`" % LIB_PATH)
_lib = ctypes.CDLL(LIB_PATH)

# ---- constants (include/lbfluct.h) ------------------------------------------------
LB_OK = 0
LB_ERR_ARG, LB_ERR_CUDA, LB_ERR_WORKSPACE = -1, -2, -3
LB_ERR_NONPOSITIVE_DENSITY, LB_ERR_NOISE_NOT_PD, LB_ERR_NONFINITE = -4, -5, -6
LB_ERR_UNSUPPORTED, LB_ERR_STATE, LB_ERR_IO, LB_ERR_NO_ROOT, LB_ERR_TIMEOUT = -7, -8, -9, -10, -11
LB_D2Q9, LB_D3Q19 = 0, 1
LB_MODEQ, LB_GUO = 0, 1
LB_FP64, LB_FP32_DEVIATION = 0, 1
LB_INIT_UNIFORM_NOISE, LB_INIT_FROM_RHO, LB_INIT_TANH_STRIPE, LB_INIT_FROM_DEVICE_RHO = 0, 1, 2, 3
LB_MAX_Q = 19
LB_MAX_LEVELS = 32
LB_MAX_HIST_BINS = 4096
LB_HIST_EST = 11
LB_VARIANT_COLS = VARIANT_COLS = 7
LB_FAULT_NONE, LB_FAULT_DENSITY, LB_FAULT_NOISE, LB_FAULT_NONFINITE, LB_FAULT_TIMEOUT, LB_FAULT_LAUNCH = range(6)
LB_NOALLOC_MAX_SITES = 1 << 18
Q_OF = {LB_D2Q9: 9, LB_D3Q19: 19}


class lb_system_desc(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int32), ("coupling", ctypes.c_int32),
                ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("rho_c", ctypes.c_double), ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("kappa", ctypes.c_double), ("kT", ctypes.c_double),
                ("tau", ctypes.c_double * LB_MAX_Q),
                ("seed", ctypes.c_uint64), ("system_id", ctypes.c_uint32)]


class lb_run_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("obs_every", ctypes.c_int32),
                ("sk_every", ctypes.c_int32), ("graph_chunk", ctypes.c_int32),
                ("tile", ctypes.c_int32 * 3), ("occupancy", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("hist_bins", ctypes.c_int32), ("jk_spectra", ctypes.c_int32), ("hist_range", ctypes.c_double)]


class lb_obs_level(ctypes.Structure):
    _fields_ = [("bx", ctypes.c_int32), ("by", ctypes.c_int32), ("bz", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("n", ctypes.c_double),
                ("sum_m", ctypes.c_double), ("sum_m2", ctypes.c_double),
                ("sum_abs_m", ctypes.c_double), ("sum_m4", ctypes.c_double),
                ("sum_e", ctypes.c_double), ("sum_e2", ctypes.c_double)]


class lb_obs_global(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("n_samples", ctypes.c_int64),
                ("mass0", ctypes.c_double), ("mass", ctypes.c_double),
                ("momentum", ctypes.c_double * 3), ("rho_mean", ctypes.c_double)]


_P = ctypes.c_void_p
_SIG = {
    "lb_workspace_bytes": (ctypes.c_int, [ctypes.POINTER(lb_system_desc), ctypes.c_int,
                                          ctypes.POINTER(lb_run_opts), ctypes.POINTER(ctypes.c_size_t)]),
    "lb_create": (ctypes.c_int, [ctypes.POINTER(lb_system_desc), ctypes.c_int, ctypes.POINTER(lb_run_opts),
                                 _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)]),
    "lb_init": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, _P]),
    "lb_stripe_density": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "lb_step": (ctypes.c_int, [_P, ctypes.c_int64]),
    "lb_sync": (ctypes.c_int, [_P]),
    "lb_observables": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(lb_obs_level), ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(lb_obs_global)]),
    "lb_observables_all": (ctypes.c_int, [_P, ctypes.POINTER(lb_obs_level), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int), ctypes.POINTER(lb_obs_global)]),
    "lb_derive": (ctypes.c_int, [ctypes.POINTER(lb_obs_level), ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
    "lb_histogram": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double)]),
    "lb_histogram_estimates": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_double, ctypes.c_double, _P]),
    "lb_momentum_spectra": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]),
    "lb_oz_fit": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P, ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                                 _P]),
    "lb_pt_workspace_bytes": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    "lb_pt_sums": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _P, ctypes.c_size_t,
                                  _P, _P]),
    "lb_pt_symmetric": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, _P, ctypes.c_size_t, _P, _P]),
    "lb_pt_broken": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, _P, ctypes.c_size_t, _P, _P]),
    "lb_structure_factor": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]),
    "lb_read_fields": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "lb_write_fields": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "lb_get_step": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "lb_save": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "lb_load": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "lb_kernel_launches": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "lb_inject_fault": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int64]),
    "lb_selftest_wait_timeout": (ctypes.c_int, [_P, _P]),
    "lb_kernel_variants": (ctypes.c_int, [ctypes.c_int, _P, ctypes.c_int]),
    "lb_kernel_variant": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "lb_block_moments_noalloc": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P,
                                                ctypes.c_int, ctypes.POINTER(ctypes.c_int), _P, _P]),
    "lb_destroy": (None, [_P]),
    "lb_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "lb_version": (ctypes.c_char_p, []),
}
for _name, (_res, _args) in _SIG.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args
    globals()[_name] = _fn

EXPORTED = tuple(_SIG)


class LBError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        msg = lb_status_string(status).decode()
        super().__init__("%s: %s (%d)" % (where, msg, status) if where else "%s (%d)" % (msg, status))


def check(status, where=""):
    if status != LB_OK:
        raise LBError(status, where)
    return status


# ---- marshalling helpers ---------------------------------------------------------
_LATTICE = {"D2Q9": LB_D2Q9, "D3Q19": LB_D3Q19}
_COUPLING = {"modeq": LB_MODEQ, "guo": LB_GUO}


def make_desc(systems):
    """ctypes array of lb_system_desc from a list of dicts (synth.system format)."""
    arr = (lb_system_desc * len(systems))()
    for k, s in enumerate(systems):
        d = arr[k]
        d.lattice = _LATTICE[s["lattice"]] if isinstance(s["lattice"], str) else int(s["lattice"])
        d.coupling = _COUPLING[s["coupling"]] if isinstance(s["coupling"], str) else int(s["coupling"])
        d.nx, d.ny, d.nz = int(s["nx"]), int(s["ny"]), int(s["nz"])
        d.rho_c, d.a, d.b = float(s["rho_c"]), float(s["a"]), float(s["b"])
        d.kappa, d.kT = float(s["kappa"]), float(s["kT"])
        for i, v in enumerate(s["tau"]):
            d.tau[i] = float(v)
        d.seed = int(s["seed"])
        d.system_id = int(s["system_id"])
    return arr


def make_opts(precision="fp64", obs_every=0, sk_every=0, graph_chunk=0, tile=(0, 0, 0), occupancy=0, variant=0,
              hist_bins=0, hist_range=0.0, jk_spectra=False):
    o = lb_run_opts()
    o.precision = {"fp64": LB_FP64, "fp32": LB_FP32_DEVIATION}.get(precision, precision)
    o.obs_every, o.sk_every, o.graph_chunk = int(obs_every), int(sk_every), int(graph_chunk)
    for k in range(3):
        o.tile[k] = int(tile[k])
    o.occupancy = int(occupancy)
    o.variant = int(variant)
    o.hist_bins = int(hist_bins)
    o.hist_range = float(hist_range)
    o.jk_spectra = 1 if jk_spectra else 0
    return o


def _pt_call(fn, nout, lattice, side, *args, device=None):
    """Run a perturbation-theory call in a torch-allocated workspace on the current stream."""
    import torch
    code = _LATTICE[lattice] if isinstance(lattice, str) else int(lattice)
    n = ctypes.c_size_t()
    check(lb_pt_workspace_bytes(code, int(side), ctypes.byref(n)), "lb_pt_workspace_bytes")
    dev = torch.device("cuda" if device is None else device)
    ws = torch.empty(n.value, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    out = (ctypes.c_double * nout)()
    check(fn(code, int(side), *[float(a) for a in args], _P(ws.data_ptr()), n.value, _P(stream.cuda_stream), out),
          fn.__name__)
    return list(out)


def pt_sums(lattice, side, m, kappa, device=None):
    """Lattice sums S1, S1sq, S2 at propagator mass m (lb_pt_sums)."""
    return dict(zip(("S1", "S1sq", "S2"), _pt_call(lb_pt_sums, 3, lattice, side, m, kappa, device=device)))


def pt_symmetric(lattice, side, r, u, kappa, kT, device=None):
    """Self-consistent r' of Eq. 36 (lb_pt_symmetric)."""
    out = _pt_call(lb_pt_symmetric, 5, lattice, side, r, u, kappa, kT, device=device)
    return dict(zip(("r_prime", "chi", "xi", "S1", "S2"), out))


def pt_broken(lattice, side, r, u, kappa, kT, device=None):
    """v, r_sigma and r'_sigma of Eqs. 40, 42, 43 (lb_pt_broken)."""
    out = _pt_call(lb_pt_broken, 7, lattice, side, r, u, kappa, kT, device=device)
    return dict(zip(("v", "r_sigma", "r_prime_sigma", "chi", "xi", "S1", "S1sq"), out))


def oz_fit(lattice, side, sums, counts, n_samples, kT, kmax):
    """Ornstein-Zernike fit of shell-binned C(k) (lb_oz_fit): dict(chi, xi, a, b, shells)."""
    code = _LATTICE[lattice] if isinstance(lattice, str) else int(lattice)
    s = np.ascontiguousarray(sums[:kmax], dtype=np.float64)
    c = np.ascontiguousarray(counts[:kmax], dtype=np.int64)
    out = (ctypes.c_double * 5)()
    check(lb_oz_fit(code, int(side), s.ctypes.data_as(_P), c.ctypes.data_as(_P), int(kmax), int(n_samples),
                    float(kT), out), "lb_oz_fit")
    return dict(chi=out[0], xi=out[1], a=out[2], b=out[3], shells=int(out[4]))


HIST_EST_FIELDS = ("m_max", "P_max", "chi_peak", "M_fit", "sigma2_fit", "chi_fit", "n_fit", "central",
                   "hist_abs_m", "hist_m2", "n_total")


def histogram_estimates(counts, lo, hi, vol, kT, m_cut=0.0, frac=0.2):
    """M_L and chi_L estimators of one level's histogram (lb_histogram_estimates)."""
    c = np.ascontiguousarray(counts, dtype=np.uint64)
    out = (ctypes.c_double * len(HIST_EST_FIELDS))()
    check(lb_histogram_estimates(c.ctypes.data_as(_P), c.size - 2, float(lo), float(hi), float(vol), float(kT),
                                 float(m_cut), float(frac), out), "lb_histogram_estimates")
    d = dict(zip(HIST_EST_FIELDS, list(out)))
    d["n_fit"] = int(d["n_fit"])
    d["central"] = bool(d["central"])
    return d


def kernel_variants(lattice):
    """Compiled step-kernel variants of a lattice: list of
    (x, y, z, occupancy, producer warps, staging, sites per thread)."""
    code = _LATTICE[lattice] if isinstance(lattice, str) else int(lattice)
    n = lb_kernel_variants(code, None, 0)
    if n < 0:
        raise LBError(n, "lb_kernel_variants")
    buf = (ctypes.c_int32 * (VARIANT_COLS * n))()
    lb_kernel_variants(code, buf, n)
    return [tuple(buf[VARIANT_COLS * r + k] for k in range(VARIANT_COLS)) for r in range(n)]


def stripe_density(systems):
    """The mean-field two-interface stripe density of every system (lb_stripe_density),
    concatenated in descriptor order, each [nz][ny][nx]."""
    desc = make_desc(systems)
    n = sum(s["nx"] * s["ny"] * s["nz"] for s in systems)
    out = np.empty(n, dtype=np.float64)
    check(lb_stripe_density(desc, len(systems), out.ctypes.data_as(_P)), "lb_stripe_density")
    return out


def workspace_bytes(systems, **opts):
    desc = make_desc(systems)
    o = make_opts(**opts)
    n = ctypes.c_size_t()
    check(lb_workspace_bytes(desc, len(systems), ctypes.byref(o), ctypes.byref(n)), "lb_workspace_bytes")
    return n.value


class Ensemble:
    """An lb_ctx over a torch-allocated workspace on the current CUDA stream."""

    def __init__(self, systems, device=None, stream=None, **opts):
        import torch
        self.systems = [dict(s) for s in systems]
        self.q = 9 if self.systems[0]["lattice"] in ("D2Q9", LB_D2Q9) else 19
        self._desc = make_desc(self.systems)
        self.n_sites = sum(int(s["nx"]) * int(s["ny"]) * int(s["nz"]) for s in self.systems)
        self._opts = make_opts(**opts)
        n = ctypes.c_size_t()
        check(lb_workspace_bytes(self._desc, len(systems), ctypes.byref(self._opts), ctypes.byref(n)),
              "lb_workspace_bytes")
        self.workspace_bytes = n.value
        dev = torch.device("cuda" if device is None else device)
        self.workspace = torch.empty(n.value, dtype=torch.uint8, device=dev)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        ctx = _P()
        check(lb_create(self._desc, len(systems), ctypes.byref(self._opts),
                        _P(self.workspace.data_ptr()), n.value, _P(self.stream.cuda_stream),
                        ctypes.byref(ctx)), "lb_create")
        self.ctx = ctx

    def shape(self, k):
        s = self.systems[k]
        return (int(s["nz"]), int(s["ny"]), int(s["nx"]))

    def init(self, mode=LB_INIT_UNIFORM_NOISE, amplitude=0.01, rho=None, rho_device=None):
        """rho: host densities (numpy, float64, systems concatenated); rho_device:
        the same as a contiguous float64 CUDA tensor, read on the context's stream."""
        ptr = None
        if rho is not None:
            self._rho = np.ascontiguousarray(rho, dtype=np.float64)
            ptr = self._rho.ctypes.data_as(_P)
            mode = LB_INIT_FROM_RHO
        elif rho_device is not None:
            import torch
            if rho_device.dtype != torch.float64 or not rho_device.is_cuda or not rho_device.is_contiguous():
                raise ValueError("rho_device: a contiguous float64 CUDA tensor")
            if rho_device.numel() != self.n_sites:
                raise ValueError("rho_device: %d values for %d sites" % (rho_device.numel(), self.n_sites))
            ptr = _P(rho_device.data_ptr())
            mode = LB_INIT_FROM_DEVICE_RHO
        check(lb_init(self.ctx, mode, float(amplitude), ptr), "lb_init")

    def step(self, n):
        check(lb_step(self.ctx, int(n)), "lb_step")

    def sync(self):
        check(lb_sync(self.ctx), "lb_sync")

    def get_step(self):
        v = ctypes.c_int64()
        check(lb_get_step(self.ctx, ctypes.byref(v)), "lb_get_step")
        return v.value

    def observables(self, k):
        lv = (lb_obs_level * LB_MAX_LEVELS)()
        n = ctypes.c_int()
        g = lb_obs_global()
        check(lb_observables(self.ctx, k, lv, LB_MAX_LEVELS, ctypes.byref(n), ctypes.byref(g)), "lb_observables")
        levels = []
        for l in range(n.value):
            L = lv[l]
            levels.append(dict(block=(L.bx, L.by, L.bz), n=L.n, sum_m=L.sum_m, sum_m2=L.sum_m2,
                               sum_abs_m=L.sum_abs_m, sum_m4=L.sum_m4, sum_e=L.sum_e, sum_e2=L.sum_e2))
        glob = dict(step=g.step, n_samples=g.n_samples, mass0=g.mass0, mass=g.mass,
                    momentum=tuple(g.momentum), rho_mean=g.rho_mean)
        return levels, glob

    def observables_all_raw(self):
        """The lb_obs_level / lb_obs_global records of every system, read with one
        copy and one synchronisation: (levels, first, globals) as ctypes arrays,
        levels[first[k]:first[k + 1]] belonging to system k."""
        n = len(self.systems)
        first = (ctypes.c_int * (n + 1))()
        check(lb_observables_all(self.ctx, None, 0, first, None), "lb_observables_all")
        total = first[n]
        lv = (lb_obs_level * max(total, 1))()
        gl = (lb_obs_global * n)()
        check(lb_observables_all(self.ctx, lv, total, first, gl), "lb_observables_all")
        return lv, first, gl

    def observables_all(self, raw=None):
        """[(levels, global)] for every system (from observables_all_raw, or a
        record of it taken earlier)."""
        n = len(self.systems)
        lv, first, gl = raw if raw is not None else self.observables_all_raw()
        out = []
        for k in range(n):
            levels = []
            for l in range(first[k], first[k + 1]):
                L = lv[l]
                levels.append(dict(block=(L.bx, L.by, L.bz), n=L.n, sum_m=L.sum_m, sum_m2=L.sum_m2,
                                   sum_abs_m=L.sum_abs_m, sum_m4=L.sum_m4, sum_e=L.sum_e, sum_e2=L.sum_e2))
            g = gl[k]
            out.append((levels, dict(step=g.step, n_samples=g.n_samples, mass0=g.mass0, mass=g.mass,
                                     momentum=tuple(g.momentum), rho_mean=g.rho_mean)))
        return out

    def derive(self, level, kT):
        L = lb_obs_level()
        L.bx, L.by, L.bz = level["block"]
        for f in ("n", "sum_m", "sum_m2", "sum_abs_m", "sum_m4", "sum_e", "sum_e2"):
            setattr(L, f, level[f])
        out = (ctypes.c_double * 6)()
        check(lb_derive(ctypes.byref(L), float(kT), out), "lb_derive")
        return dict(M_L=out[0], chi_L=out[1], chi_L_lowT=out[2], c_HL=out[3], U_L=out[4], mean_m=out[5])

    def histogram(self, k, level):
        """(counts [under, bins, over], lo, hi) of level ``level`` of system ``k``."""
        n = int(self._opts.hist_bins) + 2
        out = np.zeros(n, dtype=np.uint64)
        lo, hi = ctypes.c_double(), ctypes.c_double()
        check(lb_histogram(self.ctx, k, level, out.ctypes.data_as(_P), n, ctypes.byref(lo), ctypes.byref(hi)),
              "lb_histogram")
        return out, lo.value, hi.value

    def structure_factor(self, k, nbins):
        s = np.zeros(nbins)
        c = np.zeros(nbins, dtype=np.int64)
        ns = ctypes.c_int64()
        check(lb_structure_factor(self.ctx, k, s.ctypes.data_as(_P), c.ctypes.data_as(_P), nbins,
                                  ctypes.byref(ns)), "lb_structure_factor")
        return s, c, ns.value

    def momentum_spectra(self, k, nbins):
        """(sums (3, nbins): x, longitudinal, transverse; counts; samples) of system ``k``."""
        s = np.zeros(3 * nbins)
        c = np.zeros(nbins, dtype=np.int64)
        ns = ctypes.c_int64()
        check(lb_momentum_spectra(self.ctx, k, s.ctypes.data_as(_P), c.ctypes.data_as(_P), nbins,
                                  ctypes.byref(ns)), "lb_momentum_spectra")
        return s.reshape(3, nbins), c, ns.value

    def read_fields(self, k):
        out = np.empty((self.q,) + self.shape(k), dtype=np.float64)
        check(lb_read_fields(self.ctx, k, out.ctypes.data_as(_P)), "lb_read_fields")
        return out

    def write_fields(self, k, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (self.q,) + self.shape(k)
        check(lb_write_fields(self.ctx, k, f.ctypes.data_as(_P)), "lb_write_fields")

    def kernel_variant(self):
        """The row of kernel_variants() this context's step kernel runs."""
        v = ctypes.c_int()
        check(lb_kernel_variant(self.ctx, ctypes.byref(v)), "lb_kernel_variant")
        return v.value

    def kernel_launches(self):
        v = ctypes.c_int64()
        check(lb_kernel_launches(self.ctx, ctypes.byref(v)), "lb_kernel_launches")
        return v.value

    def save(self, path):
        check(lb_save(self.ctx, os.fsencode(path)), "lb_save")

    def load(self, path):
        check(lb_load(self.ctx, os.fsencode(path)), "lb_load")

    def close(self):
        if getattr(self, "ctx", None):
            lb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
