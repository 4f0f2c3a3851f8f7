"""Thin ctypes binding of the C ABI in include/siminf_gpu.h.

Argument marshalling only: every step of the simulation runs in the CUDA
kernels of ``libsiminf_gpu.so``.  Device buffers are torch tensors (torch is
used for device memory and streams).  There is no CPU fallback: if the
library is missing, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_PKG)
_CSRC = os.path.join(_PKG, "csrc")
_INCLUDE = os.path.join(_ROOT, "include")
_BUILD = os.path.join(_PKG, "_build")
LIB_PATH = os.path.join(_BUILD, "libsiminf_gpu.so")

SOURCES = ["sg_engine.cu", "sg_plan.cpp", "sg_mlp.cu", "sg_mparse.cpp"]
HEADERS = ["sg_common.h", "sg_device.cuh", "sg_kernels.cuh", "sg_plan.h", "sg_mlp.h", "sg_tc.cuh",
           "sg_mparse.h"]
# The headers the run-time compiler (NVRTC) sees for a model from transition
# strings, embedded into the library; NVRTC has no C library, so the two
# standard headers they include are replaced by minimal ones.
JIT_HEADERS = [("siminf_gpu.h", "include"), ("sg_common.h", "csrc"), ("sg_device.cuh", "csrc"),
               ("sg_kernels.cuh", "csrc")]
_JIT_STDINT = """#pragma once
typedef signed char int8_t;
typedef unsigned char uint8_t;
typedef short int16_t;
typedef unsigned short uint16_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long int64_t;
typedef unsigned long uint64_t;
typedef unsigned long uintptr_t;
"""
_JIT_STDDEF = """#pragma once
typedef unsigned long size_t;
"""
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", ARCH,
              "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off", "-Xcompiler", "-pthread",
              "-I" + _INCLUDE, "-I" + _CSRC, "-I" + _BUILD]

OK = 0
ERR_NAMES = {0: "ok", -1: "invalid argument",
             -2: "event moves more individuals than exist",
             -3: "shift moves outside the compartments",
             -4: "negative or non-finite transition rate",
             -5: "post time step error", -6: "device wait timed out",
             -7: "CUDA runtime error", -8: "out of memory",
             -9: "more than 2^24 draws in one node-day",
             -10: "problem exceeds the fixed scratch of sg_run_noalloc",
             -11: "transition string does not parse",
             -12: "run-time compilation or loading failed"}


class SimInfError(RuntimeError):
    def __init__(self, code, err=None):
        self.code = code
        self.err = err or {}
        super().__init__(f"siminf_gpu error {code}: {ERR_NAMES.get(code, '?')} {self.err}")


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _write_jit_sources():
    """_build/sg_jit_sources.inc: names and texts of the headers NVRTC sees."""
    names, texts = ["stdint.h", "stddef.h"], [_JIT_STDINT, _JIT_STDDEF]
    for name, where in JIT_HEADERS:
        d = _INCLUDE if where == "include" else _CSRC
        with open(os.path.join(d, name)) as f:
            names.append(name)
            texts.append(f.read())
    out = ["// generated by binding.build(): the kernel headers for NVRTC"]
    out.append("static const char *const kJitNames[] = {"
               + ", ".join('"%s"' % n for n in names) + "};")
    for i, t in enumerate(texts):
        assert ')SGSRC"' not in t
        out.append('static const char kJitSrc%d[] = R"SGSRC(%s)SGSRC";' % (i, t))
    out.append("static const char *const kJitSources[] = {"
               + ", ".join("kJitSrc%d" % i for i in range(len(texts))) + "};")
    path = os.path.join(_BUILD, "sg_jit_sources.inc")
    text = "\n".join(out) + "\n"
    if not os.path.exists(path) or open(path).read() != text:
        with open(path, "w") as f:
            f.write(text)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the CUDA library for sm_103a into ``_build/libsiminf_gpu.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    deps = ([os.path.join(_CSRC, s) for s in SOURCES + HEADERS]
            + [os.path.join(_INCLUDE, "siminf_gpu.h")])
    newest = max(os.path.getmtime(p) for p in deps)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    nvcc = _nvcc()
    objs = []
    _write_jit_sources()

    def compile_one(src):
        obj = os.path.join(_BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, "-c", os.path.join(_CSRC, src), "-o", obj] + NVCC_FLAGS
        if verbose:
            print(" ".join(cmd))
        subprocess.run(cmd, check=True)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB_PATH + ".tmp%d" % os.getpid()
    cmd = [nvcc, "-shared", ARCH, "-o", tmp] + objs + ["-Xcompiler", "-fPIC", "-ldl", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class _Desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n_nodes", ctypes.c_int32),
                ("n_comp", ctypes.c_int32), ("n_trans", ctypes.c_int32),
                ("S", ctypes.c_void_p), ("G", ctypes.c_void_p),
                ("n_select", ctypes.c_int32), ("E", ctypes.c_void_p),
                ("n_shift", ctypes.c_int32), ("N", ctypes.c_void_p),
                ("n_v", ctypes.c_int32), ("n_ldata", ctypes.c_int32),
                ("ldata", ctypes.c_void_p), ("n_gdata", ctypes.c_int32),
                ("gdata", ctypes.c_void_p)]


class Error(ctypes.Structure):
    _fields_ = [("code", ctypes.c_int32), ("rep", ctypes.c_int32),
                ("node", ctypes.c_int32), ("day", ctypes.c_int32),
                ("event", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [("reactions", ctypes.c_int64), ("draws", ctypes.c_int64),
                ("node_days", ctypes.c_int64),
                ("events_applied", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64),
                ("e2_waves", ctypes.c_int32), ("days", ctypes.c_int32),
                ("ms_ssa", ctypes.c_double), ("ms_e1", ctypes.c_double),
                ("ms_e2", ctypes.c_double), ("launches_ssa", ctypes.c_int64),
                ("launches_e1", ctypes.c_int64), ("launches_e2", ctypes.c_int64),
                ("ms_mlp", ctypes.c_double), ("launches_mlp", ctypes.c_int64),
                ("ms_host_plan", ctypes.c_double), ("ms_host_total", ctypes.c_double),
                ("node_days_rated", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = ["sg_model_create", "sg_set_events", "sg_run", "sg_run_host",
           "sg_model_destroy", "sg_strerror", "sg_philox_batch", "sg_log_batch",
           "sg_u01_batch", "sg_set_kernel_timing", "sg_fp64_fma_probe",
           "sg_run_noalloc", "sg_set_tuning", "sg_autotune", "sg_set_graphs",
           "sg_gemm_bf16", "sg_mlp_ce_loss", "sg_gelu_backward", "sg_transpose_bf16",
           "sg_colsum_bf16", "sg_adam_step", "sg_emu_features", "sg_emu_targets",
           "sg_emu_sample", "sg_emulator_set", "sg_set_neighbors", "sg_set_solver",
           "sg_set_output", "sg_model_create_parsed", "sg_model_tables",
           "sg_set_fused_events", "sg_set_persistent", "sg_gemm_fp8", "sg_quant_fp8_rows",
           "sg_quant_fp8_bf16", "sg_absmax_bf16", "sg_emulator_set_fp8", "sg_gemm_bf16_to_fp8",
           "sg_plan_events", "sg_emulator_set_min_rate", "sg_set_replicate_range"]

_lock = threading.Lock()
_lib = None


def lib(path: str | None = None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(
                f"CUDA library {p} is missing: build it with "
                "paper_1605_01421_gb300.binding.build() (there is no CPU fallback)")
        L = ctypes.CDLL(p)
        vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        L.sg_model_create.argtypes = [ctypes.POINTER(_Desc), ctypes.POINTER(vp)]
        L.sg_model_create.restype = ctypes.c_int
        L.sg_set_events.argtypes = [vp, i64] + [vp] * 9
        L.sg_set_events.restype = ctypes.c_int
        run_args = [vp, vp, i32, u64, i32, vp, vp, vp, vp, vp,
                    ctypes.POINTER(Stats), ctypes.POINTER(Error)]
        L.sg_run.argtypes = run_args
        L.sg_run.restype = ctypes.c_int
        L.sg_run_host.argtypes = run_args
        L.sg_run_host.restype = ctypes.c_int
        L.sg_model_destroy.argtypes = [vp]
        L.sg_model_destroy.restype = None
        L.sg_strerror.argtypes = [ctypes.c_int]
        L.sg_strerror.restype = ctypes.c_char_p
        L.sg_philox_batch.argtypes = [vp, u64, vp, i64, vp]
        L.sg_philox_batch.restype = ctypes.c_int
        L.sg_log_batch.argtypes = [vp, vp, i64, vp]
        L.sg_log_batch.restype = ctypes.c_int
        L.sg_u01_batch.argtypes = [vp, vp, i64, vp]
        L.sg_u01_batch.restype = ctypes.c_int
        L.sg_set_kernel_timing.argtypes = [vp, ctypes.c_int]
        L.sg_set_kernel_timing.restype = ctypes.c_int
        L.sg_fp64_fma_probe.argtypes = [i32, ctypes.POINTER(ctypes.c_double), vp]
        L.sg_fp64_fma_probe.restype = ctypes.c_int
        L.sg_run_noalloc.argtypes = [ctypes.POINTER(_Desc), vp, vp, i32, u64, i32, vp, vp,
                                     vp, vp, vp, ctypes.POINTER(Stats),
                                     ctypes.POINTER(Error)]
        L.sg_run_noalloc.restype = ctypes.c_int
        L.sg_set_tuning.argtypes = [vp, i32, i32]
        L.sg_set_tuning.restype = ctypes.c_int
        L.sg_set_replicate_range.argtypes = [vp, i32, i32]
        L.sg_set_replicate_range.restype = ctypes.c_int
        ip32 = ctypes.POINTER(ctypes.c_int32)
        L.sg_autotune.argtypes = [vp, vp, i32, u64, i32, vp, vp, vp, vp, vp, ip32, ip32,
                                  ctypes.POINTER(ctypes.c_double)]
        L.sg_autotune.restype = ctypes.c_int
        L.sg_set_graphs.argtypes = [vp, ctypes.c_int]
        L.sg_set_graphs.restype = ctypes.c_int
        L.sg_set_solver.argtypes = [vp, i32]
        L.sg_set_solver.restype = ctypes.c_int
        L.sg_set_output.argtypes = [vp, vp]
        L.sg_set_output.restype = ctypes.c_int
        L.sg_model_create_parsed.argtypes = [vp, i32, vp, i32, vp, vp, i32, i32, vp, i32, vp,
                                             i32, ctypes.POINTER(ctypes.c_void_p),
                                             ctypes.c_char_p, i32]
        L.sg_model_create_parsed.restype = ctypes.c_int
        L.sg_model_tables.argtypes = [vp, vp, vp]
        L.sg_model_tables.restype = ctypes.c_int
        L.sg_set_fused_events.argtypes = [vp, ctypes.c_int]
        L.sg_set_fused_events.restype = ctypes.c_int
        L.sg_set_persistent.argtypes = [vp, ctypes.c_int]
        L.sg_set_persistent.restype = ctypes.c_int
        L.sg_gemm_bf16.argtypes = [vp, i32, vp, i32, i32, i32, i32, vp, i32, vp, i32, vp,
                                   i32, vp]
        L.sg_gemm_bf16.restype = ctypes.c_int
        f32, f64 = ctypes.c_float, ctypes.c_double
        L.sg_mlp_ce_loss.argtypes = [vp, i32, vp, i32, vp, i32, vp, vp]
        L.sg_gelu_backward.argtypes = [vp, vp, i64, vp, vp]
        L.sg_transpose_bf16.argtypes = [vp, i32, i32, vp, vp]
        L.sg_colsum_bf16.argtypes = [vp, i32, i32, vp, vp]
        L.sg_adam_step.argtypes = [vp, vp, vp, vp, i64, f32, f32, f32, f32, i32, vp, vp]
        L.sg_emu_features.argtypes = [vp, vp, i64, vp, i32, f64, f64, f64, vp, vp, vp]
        L.sg_emulator_set_min_rate.argtypes = [vp, f64]
        L.sg_emulator_set_min_rate.restype = ctypes.c_int
        L.sg_emu_targets.argtypes = [vp, vp, i64, vp, vp]
        L.sg_emu_sample.argtypes = [vp, i32, vp, vp, i64, i32, u64, i32, vp, vp]
        L.sg_emulator_set.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), i32, f64,
                                      f64, ctypes.c_int]
        L.sg_gemm_fp8.argtypes = [vp, i32, vp, i32, i32, i32, i32, f32, vp, vp, i32, vp, i32,
                                  vp, i32, vp, i32, f32, vp]
        L.sg_gemm_bf16_to_fp8.argtypes = [vp, i32, vp, i32, i32, i32, i32, vp, i32, vp, i32,
                                          f32, vp]
        ip64 = ctypes.POINTER(ctypes.c_int64)
        L.sg_plan_events.argtypes = [i64, vp, vp, vp, vp, vp, i32, i32, i32, i32, ip64, vp, vp, vp,
                                     vp, vp]
        L.sg_plan_events.restype = ctypes.c_int
        L.sg_quant_fp8_rows.argtypes = [vp, i32, i32, vp, vp, vp]
        L.sg_quant_fp8_bf16.argtypes = [vp, i64, f32, vp, vp]
        L.sg_absmax_bf16.argtypes = [vp, i64, vp, vp]
        L.sg_emulator_set_fp8.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                          ctypes.POINTER(f32), ctypes.c_int]
        L.sg_set_neighbors.argtypes = [vp, vp, vp, vp]
        L.sg_set_neighbors.restype = ctypes.c_int
        for nm in ("sg_mlp_ce_loss", "sg_gelu_backward", "sg_transpose_bf16",
                   "sg_colsum_bf16", "sg_adam_step", "sg_emu_features", "sg_emu_targets",
                   "sg_emu_sample", "sg_emulator_set", "sg_gemm_fp8", "sg_quant_fp8_rows",
                   "sg_quant_fp8_bf16", "sg_absmax_bf16", "sg_emulator_set_fp8",
                   "sg_gemm_bf16_to_fp8"):
            getattr(L, nm).restype = ctypes.c_int
        _lib = L
        return L


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _colmajor(M):
    return np.ascontiguousarray(np.asarray(M, dtype=np.int32).ravel(order="F"))


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None and a.size else None


def _dev_ptr(t, dtype=None, shape=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (checked: the C ABI reads
    plain row-major buffers)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous (row-major)")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, not {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, not {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr()) if t.numel() else None


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class _Output(ctypes.Structure):
    _fields_ = [("dense", ctypes.c_int32), ("n_tspan", ctypes.c_int32),
                ("u_nnz", ctypes.c_int64), ("u_colptr", ctypes.c_void_p),
                ("u_row", ctypes.c_void_p), ("d_u_val", ctypes.c_void_p),
                ("v_nnz", ctypes.c_int64), ("v_colptr", ctypes.c_void_p),
                ("v_row", ctypes.c_void_p), ("d_v_val", ctypes.c_void_p),
                ("prev_cases", ctypes.c_uint32), ("prev_at_risk", ctypes.c_uint32),
                ("d_prev", ctypes.c_void_p)]


class Model:
    """A model handle (sg_model): tables of Sec. 3.2 plus scheduled events.

    ``w`` is any object with the attributes of ``workloads.Workload``:
    kind, S, G, E, N, gdata, ldata, n_v, u0 (for the node count) and events.
    """

    def __init__(self, w):
        if getattr(w, "generic", None) is not None:
            self._init_parsed(w)
        else:
            self._init_tables(w)
        self.dense = True
        if getattr(w, "events", None) is not None:
            self.set_events(w.events)
        if getattr(w, "neighbors", None) is not None:
            self.set_neighbors(*w.neighbors)
        if getattr(w, "solver", 0):
            self.set_solver(w.solver)

    def _init_tables(self, w):
        S, G = _colmajor(w.S), _colmajor(w.G)
        E, N = _colmajor(w.E), _colmajor(w.N)
        ldata = np.ascontiguousarray(np.asarray(w.ldata, np.float64).ravel(order="F"))
        gdata = np.ascontiguousarray(w.gdata, dtype=np.float64)
        n_nodes = int(np.asarray(w.u0).shape[-2])
        self.n_nodes, self.n_comp, self.n_v = n_nodes, int(w.S.shape[0]), int(w.n_v)
        self.n_trans = int(w.S.shape[1])
        d = _Desc(int(w.kind), n_nodes, int(w.S.shape[0]), int(w.S.shape[1]),
                  _p(S), _p(G), int(w.E.shape[1]), _p(E), int(w.N.shape[1]), _p(N),
                  int(w.n_v), int(np.asarray(w.ldata).shape[0]), _p(ldata),
                  int(gdata.size), _p(gdata))
        h = ctypes.c_void_p()
        rc = lib().sg_model_create(ctypes.byref(d), ctypes.byref(h))
        if rc:
            raise SimInfError(rc)
        self._h = h

    def _init_parsed(self, w):
        """A model from transition strings (sg_model_create_parsed): the
        library parses them and compiles the propensities with NVRTC."""
        g = w.generic

        def cstrs(items):
            arr = (ctypes.c_char_p * max(1, len(items)))()
            for i, x in enumerate(items):
                arr[i] = x.encode()
            return arr

        tr, cp, gn = cstrs(g["transitions"]), cstrs(g["compartments"]), cstrs(g["gdata_names"])
        gd = np.ascontiguousarray(w.gdata, dtype=np.float64)
        E, N = _colmajor(w.E), _colmajor(w.N)
        n_nodes = int(np.asarray(w.u0).shape[-2])
        msg = ctypes.create_string_buffer(4096)
        h = ctypes.c_void_p()
        rc = lib().sg_model_create_parsed(
            ctypes.cast(tr, ctypes.c_void_p), len(g["transitions"]),
            ctypes.cast(cp, ctypes.c_void_p), len(g["compartments"]),
            ctypes.cast(gn, ctypes.c_void_p), _p(gd), int(gd.size), n_nodes,
            _p(E), int(w.E.shape[1]), _p(N), int(w.N.shape[1]), ctypes.byref(h), msg, 4096)
        if rc:
            raise SimInfError(rc, {"message": msg.value.decode(errors="replace")})
        self._h = h
        self.n_nodes, self.n_comp, self.n_v = n_nodes, len(g["compartments"]), 0
        self.n_trans = len(g["transitions"])

    def tables(self):
        """(S, G) as the engine uses them: S (n_comp, n_trans), G (n_trans,
        n_trans) with G[k, j] = 1 when rate k is recomputed after j."""
        T = self.n_trans
        S = np.zeros(self.n_comp * T, np.int32)
        G = np.zeros(T * T, np.int32)
        rc = lib().sg_model_tables(self._h, _p(S), _p(G))
        if rc:
            raise SimInfError(rc)
        return S.reshape(T, self.n_comp).T.copy(), G.reshape(T, T).T.copy()

    def set_output(self, dense=True, n_tspan=0, u_pattern=None, u_values=None,
                   v_pattern=None, v_values=None, prevalence=None, prev_out=None):
        """Output selection (sg_set_output): dense U / V on or off, U_sparse
        and V_sparse patterns (colptr, row) with the layouts of U and V and
        their value tensors (CUDA int32 (R, nnz), float64 (R, nnz)), and the
        prevalence counters for ``prevalence = (cases, at_risk)``
        (compartment index lists) into ``prev_out`` (CUDA int64 (R, M, 4)).
        The tensors must stay alive for the runs that follow."""
        import torch
        keep = []

        def pat(p):
            if p is None:
                return 0, None, None
            cp = np.ascontiguousarray(p[0], dtype=np.int64)
            rw = _i32(p[1])
            keep.extend([cp, rw])
            return int(rw.size), _p(cp), (_p(rw) if rw.size else None)

        un, ucp, urw = pat(u_pattern)
        vn, vcp, vrw = pat(v_pattern)
        for t, n, nm in ((u_values, un, "u_values"), (v_values, vn, "v_values")):
            if n and (t is None or t.dim() != 2 or t.shape[1] != n):
                raise ValueError(f"{nm} must be a (n_rep, {n}) CUDA tensor")
        if prevalence is not None and (prev_out is None or prev_out.dim() != 3
                                       or tuple(prev_out.shape[1:]) != (int(n_tspan), 4)):
            raise ValueError(f"prev_out must be a (n_rep, {int(n_tspan)}, 4) CUDA tensor")
        cm = rm = 0
        if prevalence is not None:
            for c in prevalence[0]:
                cm |= 1 << int(c)
            for c in prevalence[1]:
                rm |= 1 << int(c)
        o = _Output(1 if dense else 0, int(n_tspan), un, ucp, urw,
                    _dev_ptr(u_values, torch.int32, None, "u_values") if un else None,
                    vn, vcp, vrw,
                    _dev_ptr(v_values, torch.float64, None, "v_values") if vn else None,
                    cm, rm,
                    _dev_ptr(prev_out, torch.int64, None, "prev_out") if prevalence else None)
        rc = lib().sg_set_output(self._h, ctypes.byref(o))
        if rc:
            raise SimInfError(rc)
        self._out_refs = (u_values, v_values, prev_out)
        self.dense = bool(dense)

    def set_persistent(self, enable=True):
        """One cooperative launch for the whole run when it fits (default),
        else day and E2 kernels; results are identical."""
        rc = lib().sg_set_persistent(self._h, 1 if enable else 0)
        if rc:
            raise SimInfError(rc)

    def set_fused_events(self, enable=True):
        """External transfers inside the day kernel (default) or in their
        own kernel; results are identical."""
        rc = lib().sg_set_fused_events(self._h, 1 if enable else 0)
        if rc:
            raise SimInfError(rc)

    def set_solver(self, solver):
        """0: split-step direct SSA ('ssm'), 1: all events method ('aem')."""
        rc = lib().sg_set_solver(self._h, int(solver))
        if rc:
            raise SimInfError(rc)

    def set_neighbors(self, ptr, idx, dist):
        ptr = np.ascontiguousarray(ptr, dtype=np.int64)
        idx = _i32(idx)
        dist = np.ascontiguousarray(dist, dtype=np.float64)
        rc = lib().sg_set_neighbors(self._h, _p(ptr), _p(idx), _p(dist))
        if rc:
            raise SimInfError(rc)

    def set_events(self, ev):
        L = lib()
        n = len(ev["event"])
        arrs = [_i32(ev[k]) for k in ("event", "time", "node", "dest", "n")]
        prop = np.ascontiguousarray(ev["proportion"], dtype=np.float64)
        sel, sh = _i32(ev["select"]), _i32(ev["shift"])
        rep = _i32(ev["rep"]) if ev.get("rep") is not None else None
        rc = L.sg_set_events(self._h, n, *[_p(a) for a in arrs], _p(prop), _p(sel),
                             _p(sh), _p(rep) if rep is not None else None)
        if rc:
            raise SimInfError(rc)

    def run(self, tspan, seed, n_rep, u0, v0, U, V, stream=None, check=True):
        """Run on device tensors: u0 (R, Nn, C) int32, v0 (R, Nn, Nv) float64,
        U (R, M, Nn, C) int32, V (R, M, Nn, Nv) float64, all on the GPU."""
        import torch
        L = lib()
        ts = _i32(tspan)
        st, er = Stats(), Error()
        R, Nn, C, Nv, M = int(n_rep), self.n_nodes, self.n_comp, self.n_v, int(ts.size)
        rc = L.sg_run(self._h, _p(ts), M, int(seed), R,
                      _dev_ptr(u0, torch.int32, (R, Nn, C), "u0"),
                      _dev_ptr(v0, torch.float64, (R, Nn, Nv), "v0"),
                      _dev_ptr(U, torch.int32, (R, M, Nn, C), "U") if self.dense else None,
                      _dev_ptr(V, torch.float64, (R, M, Nn, Nv), "V") if self.dense else None,
                      _stream_handle(stream), ctypes.byref(st), ctypes.byref(er))
        if rc and check:
            raise SimInfError(rc, er.as_dict())
        return rc, st.as_dict(), er.as_dict()

    def run_host(self, tspan, seed, n_rep, u0, v0, U, V, stream=None, check=True):
        """Run on host numpy arrays (pinned memory for full copy speed)."""
        L = lib()
        ts = _i32(tspan)
        st, er = Stats(), Error()
        R, Nn, C, Nv, M = int(n_rep), self.n_nodes, self.n_comp, self.n_v, int(ts.size)
        checks = [(u0, np.int32, (R, Nn, C), "u0"), (v0, np.float64, (R, Nn, Nv), "v0")]
        if self.dense:
            checks += [(U, np.int32, (R, M, Nn, C), "U"), (V, np.float64, (R, M, Nn, Nv), "V")]
        else:
            U = V = None
        for a, dt, shp, nm in checks:
            if (a.dtype != dt or a.shape != shp or not a.flags.c_contiguous
                    or (nm in ("U", "V") and not a.flags.writeable)):
                raise ValueError(f"{nm} must be a C-contiguous {np.dtype(dt).name} array "
                                 f"of shape {shp}")
        rc = L.sg_run_host(self._h, _p(ts), M, int(seed), R,
                           _p(u0), _p(v0), _p(U) if U is not None else None,
                           _p(V) if V is not None else None, _stream_handle(stream),
                           ctypes.byref(st), ctypes.byref(er))
        if rc and check:
            raise SimInfError(rc, er.as_dict())
        return rc, st.as_dict(), er.as_dict()

    def set_replicate_range(self, rep0, rep_total):
        """Runs cover the job's global replicates rep0 .. rep0 + n_rep - 1 of
        rep_total (a shard: streams keyed by the global index, other
        replicates' events left out); (0, 0) = a whole job."""
        rc = lib().sg_set_replicate_range(self._h, int(rep0), int(rep_total))
        if rc:
            raise SimInfError(rc)

    def set_tuning(self, nodes_per_block=-1, heavy_after=-1):
        rc = lib().sg_set_tuning(self._h, int(nodes_per_block), int(heavy_after))
        if rc:
            raise SimInfError(rc)

    def autotune(self, tspan, seed, n_rep, u0, v0, U, V, stream=None):
        """Pick the fastest work split on this workload; returns
        (nodes_per_block, heavy_after, ms)."""
        ts = _i32(tspan)
        npb, ha, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        rc = lib().sg_autotune(self._h, _p(ts), int(ts.size), int(seed), int(n_rep),
                               _dev_ptr(u0), _dev_ptr(v0), _dev_ptr(U), _dev_ptr(V),
                               _stream_handle(stream), ctypes.byref(npb), ctypes.byref(ha),
                               ctypes.byref(ms))
        if rc:
            raise SimInfError(rc)
        return npb.value, ha.value, ms.value

    def set_emulator(self, emu, max_herd=2000, phi_lo=0.0, phi_hi=6.0, enable=True,
                     min_rate=0.0):
        """Let sg_run use a trained emulator (emulator.Emulator) for the
        in-range nodes (herd <= max_herd, phi_lo <= phi <= phi_hi, total
        transition rate >= min_rate per day); the emulator's tensors must
        outlive the runs."""
        vp = ctypes.c_void_p
        if enable:
            W = (vp * 4)(*[ctypes.c_void_p(t.data_ptr()) for t in emu.W16])
            b = (vp * 4)(*[ctypes.c_void_p(t.data_ptr()) for t in emu.b32])
            self._emu_ref = emu
        else:
            W = b = None
        rc = lib().sg_emulator_set(self._h, W, b, int(max_herd), float(phi_lo),
                                   float(phi_hi), 1 if enable else 0)
        if rc:
            raise SimInfError(rc)
        if enable:
            rc = lib().sg_emulator_set_min_rate(self._h, float(min_rate))
            if rc:
                raise SimInfError(rc)

    def set_emulator_fp8(self, emu, enable=True):
        """Switch the emulator's layers 2-4 to E4M3 operands (the emulator
        must be quantised: emulator.Emulator.quantize_fp8); enable=False
        returns to BF16."""
        vp = ctypes.c_void_p
        if enable:
            W8 = (vp * 3)(*[ctypes.c_void_p(t.data_ptr()) for t in emu.W8])
            sc = (vp * 3)(*[ctypes.c_void_p(t.data_ptr()) for t in emu.wscale])
            act = (ctypes.c_float * 3)(*[float(a) for a in emu.act_scale])
            self._emu_fp8_ref = emu
        else:
            W8 = sc = act = None
        rc = lib().sg_emulator_set_fp8(self._h, W8, sc, act, 1 if enable else 0)
        if rc:
            raise SimInfError(rc)

    def set_graphs(self, enable=True):
        rc = lib().sg_set_graphs(self._h, 1 if enable else 0)
        if rc:
            raise SimInfError(rc)

    def set_kernel_timing(self, enable=True):
        rc = lib().sg_set_kernel_timing(self._h, 1 if enable else 0)
        if rc:
            raise SimInfError(rc)

    def close(self):
        if getattr(self, "_h", None):
            lib().sg_model_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def simulate(w, device="cuda", seed=None, n_rep=None, stream=None, tuning=None):
    """Convenience: run a workload on the GPU and return numpy (U, V, stats).
    tuning = (nodes_per_block, heavy_after) or None for the defaults."""
    import torch
    n_rep = w.n_rep if n_rep is None else n_rep
    seed = w.seed if seed is None else seed
    m = Model(w)
    if tuning is not None:
        m.set_tuning(*tuning)
    try:
        u0 = torch.as_tensor(np.array(w.u0[:n_rep], dtype=np.int32, order="C"), device=device)
        v0 = torch.as_tensor(np.array(w.v0[:n_rep], dtype=np.float64, order="C"), device=device)
        M = len(w.tspan)
        U = torch.empty((n_rep, M, m.n_nodes, m.n_comp), dtype=torch.int32, device=device)
        V = torch.empty((n_rep, M, m.n_nodes, m.n_v), dtype=torch.float64, device=device)
        rc, st, er = m.run(w.tspan, seed, n_rep, u0, v0, U, V, stream=stream)
        return U.cpu().numpy(), V.cpu().numpy(), st
    finally:
        m.close()


def gemm_bf16(A, Bt, bias=None, act=0, out32=True, out16=False, stream=None):
    """C = act(A @ Bt.T + bias) on the tensor cores.  A (M, K) and Bt (N, K)
    are contiguous BF16 CUDA tensors; returns (C32 or None, C16 or None)."""
    import torch
    M, K = A.shape
    N = Bt.shape[0]
    C32 = torch.empty((M, N), dtype=torch.float32, device=A.device) if out32 else None
    C16 = torch.empty((M, N), dtype=torch.bfloat16, device=A.device) if out16 else None
    rc = lib().sg_gemm_bf16(
        _dev_ptr(A, torch.bfloat16, (M, K), "A"), int(K),
        _dev_ptr(Bt, torch.bfloat16, (N, K), "Bt"), int(K), int(M), int(N), int(K),
        _dev_ptr(bias, torch.float32, (N,), "bias") if bias is not None else None, int(act),
        _dev_ptr(C32) if C32 is not None else None, int(N),
        _dev_ptr(C16) if C16 is not None else None, int(N), _stream_handle(stream))
    if rc:
        raise SimInfError(rc)
    return C32, C16


def gemm_fp8(A8, a_scale, B8, b_scale, bias=None, act=0, out32=True, out16=False,
             out8_inv_scale=None, stream=None):
    """C = act(A8 @ B8.T * a_scale * b_scale[n] + bias) with E4M3 operands
    on the tensor cores.  A8 (M, K) and B8 (N, K) are contiguous uint8 CUDA
    tensors holding E4M3 bytes, b_scale (N,) FP32; returns (C32, C16, C8),
    each None unless requested (C8: E4M3 bytes of the activated value times
    out8_inv_scale)."""
    import torch
    M, K = A8.shape
    N = B8.shape[0]
    dev = A8.device
    C32 = torch.empty((M, N), dtype=torch.float32, device=dev) if out32 else None
    C16 = torch.empty((M, N), dtype=torch.bfloat16, device=dev) if out16 else None
    C8 = torch.empty((M, N), dtype=torch.uint8, device=dev) if out8_inv_scale else None
    rc = lib().sg_gemm_fp8(
        _dev_ptr(A8, torch.uint8, (M, K), "A8"), int(K),
        _dev_ptr(B8, torch.uint8, (N, K), "B8"), int(K), int(M), int(N), int(K),
        float(a_scale), _dev_ptr(b_scale, torch.float32, (N,), "b_scale"),
        _dev_ptr(bias, torch.float32, (N,), "bias") if bias is not None else None, int(act),
        _dev_ptr(C32), int(N), _dev_ptr(C16), int(N), _dev_ptr(C8), int(N),
        float(out8_inv_scale or 0.0), _stream_handle(stream))
    if rc:
        raise SimInfError(rc)
    return C32, C16, C8


def plan_events(events, n_nodes, t0, t_end, slots=1):
    """The engine's host schedule of an event table for the window of unit
    steps t0 + 1 .. t_end (sg_plan_events): dict of numpy arrays order,
    e1_day, e1_node_off, e2_wave_off, wave_ev and the counts n_e1, n_e2,
    n_waves.  Runs on the host only."""
    L = lib()
    cols = [_i32(events[k]) for k in ("event", "time", "node", "dest")]
    rep = _i32(events["rep"]) if slots > 1 else None
    n = int(cols[0].size)
    counts = (ctypes.c_int64 * 3)()
    args = [n] + [_p(c) for c in cols] + [_p(rep) if rep is not None else None,
                                          int(n_nodes), int(t0), int(t_end), int(slots)]
    rc = L.sg_plan_events(*args, counts, None, None, None, None, None)
    if rc:
        raise SimInfError(rc)
    n_e1, n_e2, n_w = (int(c) for c in counts)
    days = int(t_end) - int(t0)
    out = {"order": np.zeros(n_e1 + n_e2, np.int64), "e1_day": np.zeros(n_e1, np.int32),
           "e1_node_off": np.zeros(slots * n_nodes + 1, np.int64),
           "e2_wave_off": np.zeros(days * slots + 1, np.int64),
           "wave_ev": np.zeros(n_w + 1, np.int64)}
    rc = L.sg_plan_events(*args, counts, *[_p(out[k]) for k in ("order", "e1_day", "e1_node_off",
                                                                 "e2_wave_off", "wave_ev")])
    if rc:
        raise SimInfError(rc)
    out.update(n_e1=n_e1, n_e2=n_e2, n_waves=n_w)
    return out


def gemm_bf16_to_fp8(A, Bt, inv_scale, bias=None, act=0, stream=None):
    """E4M3 bytes (uint8) of act(A @ Bt.T + bias) * inv_scale for BF16 A (M,
    K) and Bt (N, K)."""
    import torch
    M, K = A.shape
    N = Bt.shape[0]
    C8 = torch.empty((M, N), dtype=torch.uint8, device=A.device)
    rc = lib().sg_gemm_bf16_to_fp8(
        _dev_ptr(A, torch.bfloat16, (M, K), "A"), int(K),
        _dev_ptr(Bt, torch.bfloat16, (N, K), "Bt"), int(K), int(M), int(N), int(K),
        _dev_ptr(bias, torch.float32, (N,), "bias") if bias is not None else None, int(act),
        _dev_ptr(C8), int(N), float(inv_scale), _stream_handle(stream))
    if rc:
        raise SimInfError(rc)
    return C8


def quant_fp8_rows(W, stream=None):
    """Per-row E4M3 quantisation of an FP32 matrix: (W8 uint8, scale FP32)
    with W ~ W8 * scale[:, None]."""
    import torch
    rows, cols = W.shape
    W8 = torch.empty((rows, cols), dtype=torch.uint8, device=W.device)
    sc = torch.empty((rows,), dtype=torch.float32, device=W.device)
    rc = lib().sg_quant_fp8_rows(_dev_ptr(W, torch.float32, (rows, cols), "W"), int(rows),
                                 int(cols), _dev_ptr(W8), _dev_ptr(sc), _stream_handle(stream))
    if rc:
        raise SimInfError(rc)
    return W8, sc


def quant_fp8_bf16(x, inv_scale, stream=None):
    """E4M3 bytes of x * inv_scale for a BF16 tensor x."""
    import torch
    out = torch.empty(x.shape, dtype=torch.uint8, device=x.device)
    rc = lib().sg_quant_fp8_bf16(_dev_ptr(x, torch.bfloat16), x.numel(), float(inv_scale),
                                 _dev_ptr(out), _stream_handle(stream))
    if rc:
        raise SimInfError(rc)
    return out


def absmax_bf16(x, stream=None):
    """max |x| of a BF16 tensor, as a Python float."""
    import torch
    out = torch.zeros((1,), dtype=torch.float32, device=x.device)
    rc = lib().sg_absmax_bf16(_dev_ptr(x, torch.bfloat16), x.numel(), _dev_ptr(out),
                              _stream_handle(stream))
    if rc:
        raise SimInfError(rc)
    return float(out.item())


def fp64_fma_probe(iters=20000, stream=None):
    """Measured FP64 fused multiply-add throughput of this GPU, TFLOP/s."""
    out = ctypes.c_double()
    rc = lib().sg_fp64_fma_probe(int(iters), ctypes.byref(out), _stream_handle(stream))
    if rc:
        raise SimInfError(rc)
    return out.value


def philox_batch(ctr, key, stream=None):
    import torch
    c = torch.as_tensor(np.ascontiguousarray(ctr, dtype=np.uint32).view(np.int32),
                        device="cuda")
    out = torch.empty_like(c)
    rc = lib().sg_philox_batch(_dev_ptr(c), int(key), _dev_ptr(out), c.numel() // 4,
                               _stream_handle(stream))
    if rc:
        raise SimInfError(rc)
    return out.cpu().numpy().view(np.uint32)


def log_batch(x, stream=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")
    y = torch.empty_like(t)
    rc = lib().sg_log_batch(_dev_ptr(t), _dev_ptr(y), t.numel(), _stream_handle(stream))
    if rc:
        raise SimInfError(rc)
    return y.cpu().numpy()


def u01_batch(words, stream=None):
    import torch
    w = torch.as_tensor(np.ascontiguousarray(words, dtype=np.uint32).view(np.int32),
                        device="cuda")
    y = torch.empty(w.numel() // 2, dtype=torch.float64, device="cuda")
    rc = lib().sg_u01_batch(_dev_ptr(w), _dev_ptr(y), y.numel(), _stream_handle(stream))
    if rc:
        raise SimInfError(rc)
    return y.cpu().numpy()
