"""Thin Python binding of the ILVES C ABI (``include/ilves.h``).

Argument marshalling only: torch tensors are checked (device, dtype, layout) and
their device pointers handed to ``libilves.so``; every step of the solve runs in
the library's CUDA kernels.  There is no CPU fallback: without the built library
every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libilves.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "ilves.h")

FP64, MIXED, MIXED_DF = 0, 1, 2
CHORD = 256  # ILVES-F flag
START_DIAG = 512  # diagonal starting multipliers computed inside the solve
PRECISIONS = {"fp64": FP64, "mixed": MIXED, "mixed_df": MIXED_DF}
CONVERGED, MAX_ITER, SINGULAR_PIVOT, NONFINITE, WAIT_TIMEOUT = 0, 1, 2, 3, 4
STATUS = {0: "ok", 1: "invalid argument", 2: "invalid topology", 3: "CUDA error", 4: "out of device memory",
          5: "device wait timed out", 6: "scratch needed exceeds the static maximum"}


class IlvesError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"{where}: {STATUS.get(code, code)} (status {code})")
        self.code = code


class SetupOpts(ctypes.Structure):
    _fields_ = [("ordering", ctypes.c_int32), ("degree_slack", ctypes.c_int32),
                ("warps_per_cta", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("device", ctypes.c_int32), ("max_warp_constraints", ctypes.c_int32),
                ("partition_min_constraints", ctypes.c_int32), ("part_constraints", ctypes.c_int32),
                ("wait_test", ctypes.c_int32), ("overlap", ctypes.c_int32), ("narrow_atoms", ctypes.c_int32)]


class Tuning(ctypes.Structure):
    _fields_ = [("chosen", SetupOpts), ("candidates", ctypes.c_int32), ("best_ms", ctypes.c_float),
                ("before_ms", ctypes.c_float)]


_lib = None


def lib():
    """The loaded C library; raises if it was not built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"ILVES CUDA library missing at {LIB_PATH}; build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    P, I32, I64, D, VP = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
    pi32 = ctypes.POINTER(I32)
    pi64 = ctypes.POINTER(I64)
    L.ilves_default_opts.argtypes = [ctypes.POINTER(SetupOpts)]
    L.ilves_default_opts.restype = None
    L.ilves_setup_topology.argtypes = [I32, I32, P, P, ctypes.POINTER(SetupOpts), ctypes.POINTER(P)]
    L.ilves_setup_topology.restype = I32
    L.ilves_solve.argtypes = [P, P, P, P, P, D, I32, I32, P, P, P, P, P, VP]
    L.ilves_solve.restype = I32
    L.ilves_topology_info.argtypes = [P, pi32, pi64, pi32, pi64, pi32]
    L.ilves_topology_info.restype = I32
    L.ilves_topology_molecules.argtypes = [P, P, P, P, P]
    L.ilves_topology_molecules.restype = I32
    L.ilves_topology_export_molecule.argtypes = [P, I32, P, P, P, P]
    L.ilves_topology_export_molecule.restype = I32
    L.ilves_autotune.argtypes = [P, P, P, P, P, D, I32, I32, VP, ctypes.POINTER(Tuning)]
    L.ilves_autotune.restype = I32
    L.ilves_topology_tuning.argtypes = [P, ctypes.POINTER(Tuning)]
    L.ilves_topology_tuning.restype = I32
    L.ilves_topology_export_domains.argtypes = [P, I32, P, P, P, P, P]
    L.ilves_topology_export_domains.restype = I32
    L.ilves_topology_export_layout.argtypes = [P, I32, P, P, P, P, P]
    L.ilves_topology_export_layout.restype = I32
    L.ilves_topology_schedule.argtypes = [P, I32, I32, I32, P, P, P, P, P, P, P, P, P, P]
    L.ilves_topology_schedule.restype = I32
    L.ilves_destroy_topology.argtypes = [P]
    L.ilves_destroy_topology.restype = None
    L.ilves_status_string.argtypes = [I32]
    L.ilves_status_string.restype = ctypes.c_char_p
    L.ilves_last_launch_count.argtypes = [P]
    L.ilves_last_launch_count.restype = I32
    L.ilves_solve_static_scratch.argtypes = [P, P, P, P, P, D, I32, I32, P, P, P, P, P, VP]
    L.ilves_solve_static_scratch.restype = I32
    L.ilves_static_scratch_bytes.argtypes = []
    L.ilves_static_scratch_bytes.restype = I64
    L.ilves_topology_workspace_bytes.argtypes = [P]
    L.ilves_topology_workspace_bytes.restype = I64
    L.ilves_topology_device_bytes.argtypes = [P]
    L.ilves_topology_device_bytes.restype = I64
    L.ilves_measure_fp64_fma.argtypes = [I32, ctypes.POINTER(D), VP]
    L.ilves_measure_fp64_fma.restype = I32
    L.ilves_mlp_param_count.argtypes = []
    L.ilves_mlp_param_count.restype = I64
    L.ilves_mlp_check.argtypes = [P, pi32]
    L.ilves_mlp_check.restype = I32
    L.ilves_mlp_set_wait_test.argtypes = [P, I32]
    L.ilves_mlp_set_wait_test.restype = I32
    L.ilves_mlp_create.argtypes = [I32, ctypes.c_uint64, ctypes.POINTER(P)]
    L.ilves_mlp_create.restype = I32
    L.ilves_mlp_destroy.argtypes = [P]
    L.ilves_mlp_destroy.restype = None
    for n in ("ilves_mlp_set_params", "ilves_mlp_get_params"):
        getattr(L, n).argtypes = [P, P]
        getattr(L, n).restype = I32
    L.ilves_mlp_features.argtypes = [P, P, P, P, P, P, P, VP]
    L.ilves_mlp_features.restype = I32
    L.ilves_mlp_forward.argtypes = [P, P, I32, P, VP]
    L.ilves_mlp_forward.restype = I32
    L.ilves_warm_start.argtypes = [P, P, P, P, P, P, P, VP]
    L.ilves_warm_start.restype = I32
    L.ilves_mlp_gradient.argtypes = [P, P, P, I32, P, P, VP]
    L.ilves_mlp_gradient.restype = I32
    L.ilves_mlp_train_step.argtypes = [P, P, P, I32, ctypes.c_float, P, VP]
    L.ilves_mlp_train_step.restype = I32
    _lib = L
    return L


def header_functions():
    """Names of the functions ``include/ilves.h`` declares."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ilves_[a-z_]+)\s*\(", src)))


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if isinstance(a, np.ndarray) else ctypes.c_void_p(a.data_ptr())


def _check(code, where):
    if code != 0:
        raise IlvesError(code, where)


class Topology:
    """A constraint topology set up once and solved many times (``ilves_setup_topology``)."""

    def __init__(self, n_atoms, atom_i, atom_j, ordering=0, degree_slack=2, warps_per_cta=0,
                 ctas_per_sm=0, device=None, plan_only=False, max_warp_constraints=0,
                 partition_min_constraints=0, part_constraints=0, wait_test=0, overlap=0, narrow_atoms=0):
        L = lib()
        ai = np.ascontiguousarray(atom_i, dtype=np.int32)
        aj = np.ascontiguousarray(atom_j, dtype=np.int32)
        if ai.shape != aj.shape or ai.ndim != 1:
            raise ValueError("atom_i and atom_j must be 1-D arrays of equal length")
        o = SetupOpts()
        L.ilves_default_opts(ctypes.byref(o))
        o.ordering, o.degree_slack = ordering, degree_slack
        o.warps_per_cta, o.ctas_per_sm = warps_per_cta, ctas_per_sm
        o.max_warp_constraints = max_warp_constraints
        o.partition_min_constraints = partition_min_constraints
        o.part_constraints = part_constraints
        o.wait_test = wait_test
        o.overlap = overlap
        o.narrow_atoms = narrow_atoms
        if plan_only:
            o.device = -2
        elif device is not None:
            o.device = int(device)
        h = ctypes.c_void_p()
        _check(L.ilves_setup_topology(int(n_atoms), ai.size, _ptr(ai), _ptr(aj), ctypes.byref(o), ctypes.byref(h)),
               "ilves_setup_topology")
        self._h = h
        self.n_atoms = int(n_atoms)
        self.n_constraints = int(ai.size)
        self.plan_only = plan_only
        self._device_index = None if device is None else int(device)
        self._refresh_info()

    def _refresh_info(self):
        n = ctypes.c_int32()
        nnz = ctypes.c_int64()
        ml = ctypes.c_int32()
        fill = ctypes.c_int64()
        nl = ctypes.c_int32()
        _check(lib().ilves_topology_info(self._h, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(ml),
                                         ctypes.byref(fill), ctypes.byref(nl)), "ilves_topology_info")
        self.n_molecules, self.nnz_factor, self.max_levels = n.value, nnz.value, ml.value
        self.n_fill, self.n_large = fill.value, nl.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().ilves_destroy_topology(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def molecules(self):
        """Per-molecule (atoms, constraints, levels, first_atom) as int32 numpy arrays."""
        n = self.n_molecules
        out = [np.zeros(n, np.int32) for _ in range(4)]
        _check(lib().ilves_topology_molecules(self._h, *[_ptr(a) for a in out]), "ilves_topology_molecules")
        return tuple(out)

    def export_molecule(self, mol):
        """(pos_gid, level, up_ptr, up_idx) of one molecule's symbolic factorisation."""
        atoms, cons, _, _ = self.molecules()
        nc = int(cons[mol])
        pos = np.zeros(nc, np.int32)
        lev = np.zeros(nc, np.int32)
        ptr = np.zeros(nc + 1, np.int32)
        L = lib()
        _check(L.ilves_topology_export_molecule(self._h, int(mol), _ptr(pos), _ptr(lev), _ptr(ptr), None),
               "export")
        idx = np.zeros(max(1, int(ptr[-1])), np.int32)
        _check(L.ilves_topology_export_molecule(self._h, int(mol), None, None, None, _ptr(idx)), "export")
        return pos, lev, ptr, idx[: ptr[-1]]

    def export_layout(self, mol):
        """``ilves_topology_export_layout``: dict with the global atom of each local atom
        (``atom_gid``), and for a partitioned molecule the parts' levels and program bytes and
        the separator block's levels, program bytes, interior terms and the largest part
        program (bytes, with its scratch area)."""
        atoms, _, _, _ = self.molecules()
        L = lib()
        na = int(atoms[mol])
        gid = np.zeros(max(1, na), np.int32)
        n_parts = ctypes.c_int32()
        _check(L.ilves_topology_export_layout(self._h, int(mol), _ptr(gid), ctypes.byref(n_parts), None, None, None),
               "export_layout")
        npart = n_parts.value
        lev = np.zeros(max(1, npart), np.int32)
        pb = np.zeros(max(1, npart), np.int32)
        sep = np.zeros(4, np.int32)
        _check(L.ilves_topology_export_layout(self._h, int(mol), None, None, _ptr(lev), _ptr(pb), _ptr(sep)),
               "export_layout")
        return {"atom_gid": gid[:na], "n_parts": npart, "part_levels": lev[:npart], "part_prog_bytes": pb[:npart],
                "sep_levels": int(sep[0]), "sep_prog_bytes": int(sep[1]), "sep_interior_terms": int(sep[2]),
                "part_prog_max": int(sep[3])}

    @staticmethod
    def _tuning_dict(t):
        c = t.chosen
        return {"candidates": t.candidates, "best_ms": t.best_ms, "before_ms": t.before_ms,
                "chosen": {f: getattr(c, f) for f, _ in SetupOpts._fields_ if f not in ("device", "wait_test")}}

    def autotune(self, x_old, x_unc, inv_mass, d, tol=1e-12, precision="mixed", start=None, reps=5, stream=None):
        """``ilves_autotune``: time candidate set-up options on these inputs and keep the fastest
        (the topology is re-planned in place); returns the tuning as a dict."""
        import torch

        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        if start == "diag":
            prec |= START_DIAG
        t = Tuning()
        s = torch.cuda.current_stream(x_unc.device if x_unc.is_cuda else None).cuda_stream if stream is None \
            else stream.cuda_stream
        _check(lib().ilves_autotune(self._h, _ptr(x_old), _ptr(x_unc), _ptr(inv_mass), _ptr(d), float(tol), prec,
                                    int(reps), ctypes.c_void_p(s), ctypes.byref(t)), "ilves_autotune")
        self._refresh_info()
        return self._tuning_dict(t)

    def tuning(self):
        """``ilves_topology_tuning``: the last autotuning (candidates == 0: never tuned)."""
        t = Tuning()
        _check(lib().ilves_topology_tuning(self._h, ctypes.byref(t)), "ilves_topology_tuning")
        return self._tuning_dict(t)

    def export_domains(self, mol=0):
        """``ilves_topology_export_domains``: overlapping domains of one molecule as a dict with
        atom_bounds (n_dom + 1), and per domain d its constraints' global ids cons[d] and owned
        flags owned[d] (numpy arrays); empty lists if the molecule is not solved by domains."""
        L = lib()
        nd = ctypes.c_int32()
        _check(L.ilves_topology_export_domains(self._h, int(mol), ctypes.byref(nd), None, None, None, None),
               "export_domains")
        n = nd.value
        if n == 0:
            return {"atom_bounds": np.zeros(0, np.int32), "cons": [], "owned": []}
        bounds = np.zeros(n + 1, np.int32)
        ptr = np.zeros(n + 1, np.int32)
        _check(L.ilves_topology_export_domains(self._h, int(mol), None, _ptr(bounds), _ptr(ptr), None, None),
               "export_domains")
        gid = np.zeros(max(1, int(ptr[-1])), np.int32)
        own = np.zeros(max(1, int(ptr[-1])), np.int32)
        _check(L.ilves_topology_export_domains(self._h, int(mol), None, None, None, _ptr(gid), _ptr(own)),
               "export_domains")
        return {"atom_bounds": bounds, "cons": [gid[ptr[d]:ptr[d + 1]] for d in range(n)],
                "owned": [own[ptr[d]:ptr[d + 1]].astype(bool) for d in range(n)]}

    def schedule(self, precision="mixed", n_cta=152, arena_bytes=232448):
        """Host plan of the batched kernel's slots (``ilves_topology_schedule``): dict with
        slot_cta, slot_bytes, slot_queue, slot_team (per slot), mol_slot (slot, -1 pool, -2
        off the batched path), mol_bytes and mol_team (per molecule), pool_n, and the
        96-thread class's n_slots_wide and pool_wide, the launch's block_threads and the
        most slots of one CTA (max_slots)."""
        L = lib()
        prec = PRECISIONS[precision]
        ns, pn = ctypes.c_int32(), ctypes.c_int32()
        _check(L.ilves_topology_schedule(self._h, prec, int(n_cta), int(arena_bytes), ctypes.byref(ns),
                                         ctypes.byref(pn), *([None] * 8)), "ilves_topology_schedule")
        slot_keys = ("slot_cta", "slot_bytes", "slot_queue", "slot_team")
        mol_keys = ("mol_slot", "mol_bytes", "mol_team")
        out = {k: np.zeros(ns.value, np.int32) for k in slot_keys}
        out.update({k: np.zeros(self.n_molecules, np.int32) for k in mol_keys})
        ci = np.zeros(4, np.int32)
        _check(L.ilves_topology_schedule(self._h, prec, int(n_cta), int(arena_bytes), None, None,
                                         *[_ptr(out[k]) for k in slot_keys + mol_keys], _ptr(ci)),
               "ilves_topology_schedule")
        out["pool_n"] = pn.value
        out["n_slots_wide"], out["pool_wide"], out["block_threads"], out["max_slots"] = (int(v) for v in ci)
        return out

    def last_launch_count(self):
        return int(lib().ilves_last_launch_count(self._h))

    def device_bytes(self):
        return int(lib().ilves_topology_device_bytes(self._h))

    def workspace_bytes(self):
        return int(lib().ilves_topology_workspace_bytes(self._h))

    def solve_static_scratch(self, *args, **kw):
        """``ilves_solve_static_scratch``: as ``solve``, but the large-molecule state lives in the
        library's static device array, so the call itself allocates nothing on the device.
        (This Python wrapper still creates output tensors when none are passed.)"""
        return self.solve(*args, _entry="ilves_solve_static_scratch", **kw)

    def solve(self, x_old, x_unc, inv_mass, d, tol=1e-12, max_iter=25, precision="mixed", lambda0=None,
              x_out=None, lambda_out=None, iterations_out=None, status_out=None, stream=None,
              method="newton", start=None, _entry="ilves_solve"):
        """One ``ilves_solve``; returns (x, lambda, iterations, status).  Every tensor is a
        CUDA tensor on the topology's device or a page-locked (pinned) host tensor, which the
        kernels read or write in place; outputs not given are allocated like ``x_unc``.
        ``start="diag"`` computes the diagonal starting multipliers inside the solve
        (``ILVES_START_DIAG``; lambda0 must then be None)."""
        import torch

        if self.plan_only:
            raise RuntimeError("topology was planned on the host only")
        given = [t for t in (x_old, x_unc, inv_mass, d, lambda0, x_out, lambda_out, iterations_out, status_out)
                 if t is not None]
        dev = next((t.device for t in given if t.is_cuda), None)
        if dev is None:
            dev = torch.device("cuda", self._device_index if self._device_index is not None
                               else torch.cuda.current_device())

        def placed(t):  # on the solve's device, or page-locked host memory
            return t.device == dev or (t.device.type == "cpu" and t.is_pinned())

        for name, t, shape in (("x_old", x_old, (self.n_atoms, 3)), ("x_unc", x_unc, (self.n_atoms, 3)),
                               ("inv_mass", inv_mass, (self.n_atoms,)), ("d", d, (self.n_constraints,))):
            if t.dtype != torch.float64 or tuple(t.shape) != shape or not t.is_contiguous() or not placed(t):
                raise ValueError(f"{name} must be a contiguous float64 tensor of shape {shape}, "
                                 "on the CUDA device or in pinned host memory")
        if lambda0 is not None and (lambda0.dtype != torch.float32 or lambda0.numel() != self.n_constraints
                                    or not lambda0.is_contiguous() or not placed(lambda0)):
            raise ValueError("lambda0 must be a contiguous float32 tensor of n_constraints entries")
        host = x_unc.device.type == "cpu"

        def alloc(n, dtype):
            return torch.empty(n, dtype=dtype, pin_memory=True) if host else torch.empty(n, dtype=dtype, device=dev)

        x_out = alloc((self.n_atoms, 3), torch.float64) if x_out is None else x_out
        lambda_out = alloc(self.n_constraints, torch.float64) if lambda_out is None else lambda_out
        iterations_out = alloc(self.n_molecules, torch.int32) if iterations_out is None else iterations_out
        status_out = alloc(self.n_molecules, torch.int32) if status_out is None else status_out
        for name, t, dtype, n in (("x_out", x_out, torch.float64, 3 * self.n_atoms),
                                  ("lambda_out", lambda_out, torch.float64, self.n_constraints),
                                  ("iterations_out", iterations_out, torch.int32, self.n_molecules),
                                  ("status_out", status_out, torch.int32, self.n_molecules)):
            if t.dtype != dtype or t.numel() != n or not t.is_contiguous() or not placed(t):
                raise ValueError(f"{name} must be a contiguous {dtype} tensor of {n} entries, "
                                 "on the CUDA device or in pinned host memory")
        s = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream.cuda_stream
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        if method == "chord":
            prec |= CHORD
        elif method != "newton":
            raise ValueError("method must be 'newton' (ILVES-M) or 'chord' (ILVES-F)")
        if start == "diag":
            if lambda0 is not None:
                raise ValueError("start='diag' computes lambda0 itself; pass lambda0=None")
            prec |= START_DIAG
        elif start is not None:
            raise ValueError("start must be None or 'diag'")
        fn = getattr(lib(), _entry)
        _check(fn(self._h, _ptr(x_old), _ptr(x_unc), _ptr(inv_mass), _ptr(d), float(tol), int(max_iter),
                  prec, None if lambda0 is None else _ptr(lambda0), _ptr(x_out), _ptr(lambda_out),
                  _ptr(iterations_out), _ptr(status_out), ctypes.c_void_p(s)), _entry)
        return x_out, lambda_out, iterations_out, status_out


def measure_fp64_fma(iters=4096, stream=None, device=None):
    """``ilves_measure_fp64_fma``: the float64 FMA rate of the current device, GFLOP/s."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    g = ctypes.c_double()
    _check(lib().ilves_measure_fp64_fma(int(iters), ctypes.byref(g), _stream(dev, stream)), "ilves_measure_fp64_fma")
    return g.value


def _stream(dev, stream=None):
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream if stream is None else stream.cuda_stream)


def _check_tensor(name, t, dtype, numel):
    import torch

    if t.dtype != dtype or t.numel() != numel or not t.is_contiguous() or t.device.type != "cuda":
        raise ValueError(f"{name} must be a contiguous {dtype} CUDA tensor with {numel} elements")


class Mlp:
    """The warm-start network (``ilves_mlp_*``): 16 -> 128 -> 128 -> 1, bfloat16 weights."""

    N_FEATURES = 16

    def __init__(self, max_batch=65536, seed=0):
        L = lib()
        h = ctypes.c_void_p()
        _check(L.ilves_mlp_create(int(max_batch), ctypes.c_uint64(seed), ctypes.byref(h)), "ilves_mlp_create")
        self._h = h
        self.max_batch = int(max_batch)
        self.n_params = int(L.ilves_mlp_param_count())

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().ilves_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self):
        """Number of tensor-core waits that gave up (synchronises; 0 in a healthy run)."""
        n = ctypes.c_int32()
        lib().ilves_mlp_check(self._h, ctypes.byref(n))
        return n.value

    def set_wait_test(self, on):
        """Testing only (``ilves_mlp_set_wait_test``): forward kernels wait on a barrier nothing
        signals, so the bounded wait runs out and ``check()`` reports it."""
        _check(lib().ilves_mlp_set_wait_test(self._h, 1 if on else 0), "ilves_mlp_set_wait_test")

    def get_params(self):
        out = np.zeros(self.n_params, np.float32)
        _check(lib().ilves_mlp_get_params(self._h, _ptr(out)), "ilves_mlp_get_params")
        return out

    def set_params(self, theta):
        a = np.ascontiguousarray(theta, dtype=np.float32)
        if a.size != self.n_params:
            raise ValueError("wrong parameter count")
        _check(lib().ilves_mlp_set_params(self._h, _ptr(a)), "ilves_mlp_set_params")

    def save(self, path):
        np.save(path, self.get_params())

    def load(self, path):
        self.set_params(np.load(path))

    def forward(self, features, stream=None):
        import torch

        n = features.shape[0]
        _check_tensor("features", features, torch.float32, n * self.N_FEATURES)
        y = torch.empty(n, dtype=torch.float32, device=features.device)
        _check(lib().ilves_mlp_forward(self._h, _ptr(features), n, _ptr(y), _stream(features.device, stream)),
               "ilves_mlp_forward")
        return y

    def gradient(self, features, target, stream=None):
        import torch

        n = features.shape[0]
        _check_tensor("features", features, torch.float32, n * self.N_FEATURES)
        _check_tensor("target", target, torch.float32, n)
        g = torch.empty(self.n_params, dtype=torch.float32, device=features.device)
        loss = torch.empty(1, dtype=torch.float32, device=features.device)
        _check(lib().ilves_mlp_gradient(self._h, _ptr(features), _ptr(target), n, _ptr(g), _ptr(loss),
                                        _stream(features.device, stream)), "ilves_mlp_gradient")
        return g, loss

    def train_step(self, features, target, lr, loss_out=None, stream=None):
        import torch

        n = features.shape[0]
        _check_tensor("features", features, torch.float32, n * self.N_FEATURES)
        _check_tensor("target", target, torch.float32, n)
        _check(lib().ilves_mlp_train_step(self._h, _ptr(features), _ptr(target), n, ctypes.c_float(lr),
                                          None if loss_out is None else _ptr(loss_out),
                                          _stream(features.device, stream)), "ilves_mlp_train_step")


def features(topo, x_old, x_unc, inv_mass, d, stream=None):
    """``ilves_mlp_features``: (features (n_c, 16) float32, scale (n_c,) float32) on the device."""
    import torch

    dev = x_unc.device
    f = torch.empty(topo.n_constraints, 16, dtype=torch.float32, device=dev)
    sc = torch.empty(topo.n_constraints, dtype=torch.float32, device=dev)
    _check(lib().ilves_mlp_features(topo._h, _ptr(x_old), _ptr(x_unc), _ptr(inv_mass), _ptr(d), _ptr(f), _ptr(sc),
                                    _stream(dev, stream)), "ilves_mlp_features")
    return f, sc


def warm_start(mlp, topo, x_old, x_unc, inv_mass, d, out=None, stream=None):
    """``ilves_warm_start``: lambda_0 (float32, n_c) from the network, or the diagonal guess if mlp is None."""
    import torch

    dev = x_unc.device
    out = torch.empty(topo.n_constraints, dtype=torch.float32, device=dev) if out is None else out
    _check(lib().ilves_warm_start(None if mlp is None else mlp._h, topo._h, _ptr(x_old), _ptr(x_unc), _ptr(inv_mass),
                                  _ptr(d), _ptr(out), _stream(dev, stream)), "ilves_warm_start")
    return out
