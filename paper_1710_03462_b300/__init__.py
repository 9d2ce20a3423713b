"""soax-b300: a Structure-of-Arrays particle container for the NVIDIA B300 (sm_103a).

Python binding of the C-ABI library libsoax.so (include/soax.h).  This module only
marshals arguments: every step of the computation runs in the library's CUDA kernels.
PyTorch provides device memory and streams.

The container follows the paper's SoAx (Sec. 4): a particle type is a list of
attributes (name, scalar type, number of components, one-character tag), stored as one
device array per component.  On top of it the library runs

  * the inertial-particle midpoint-RK2 step in the ABC flow (soax_step), generalising
    the Euler advection x += dt*v of Eq. 1 (Sec. 2), on SoA planes or AoS records;
  * the cell-key radix sort and the permute-gather of every plane (soax_sort_by_cell);
  * the AoS <-> SoA transposes (bulk getElement / push_back of Listing 6);
  * the checkpointed forward and its adjoint (SoaxRK2, a torch.autograd.Function);
  * a batched persistent step over many ensembles, with an autotuner.

There is no CPU fallback: if the library cannot be loaded, every call raises.
"""
import ast
import ctypes as C
import hashlib
import json
import os
from dataclasses import dataclass

import torch

from . import _abi
from ._abi import DTYPES, EXPR_OPS, STATUS_NAMES, soax_expr_op, soax_field_desc, soax_flow, soax_tune

__all__ = ["SoaxError", "lib", "Particles", "Flow", "Tune", "radix_sort_pairs", "step_batched", "euler_aos",
           "batched_workspace", "autotune", "sync", "SoaxRK2", "TWO_PI", "BASIC_SCHEMA", "WIDE_SCHEMA",
           "parse_expr"]

TWO_PI = 6.283185307179586

# The record of the program summary, {int id; double pos[3]; float vel[3];}, with the
# tags of Listing 5 (N identity, P position, V velocity).
BASIC_SCHEMA = [("id", "i32", 1, "N"), ("pos", "f64", 3, "P"), ("vel", "f32", 3, "V")]
# A wider heterogeneous record (acceleration, mass, a small integer tag).
WIDE_SCHEMA = [("id", "i64", 1, "N"), ("pos", "f64", 3, "P"), ("vel", "f32", 3, "V"),
               ("acc", "f32", 3, "A"), ("mass", "f32", 1, "M"), ("tag", "u8", 1, "T")]

TORCH_DTYPES = {"i32": torch.int32, "i64": torch.int64, "u8": torch.uint8, "f32": torch.float32,
                "f64": torch.float64}


_BINOPS = {ast.Add: "add", ast.Sub: "sub", ast.Mult: "mul", ast.Div: "div"}
_CALLS = {"sqrt": ("sqrt", 1), "abs": ("abs", 1), "min": ("min", 2), "max": ("max", 2), "fma": ("fma", 3)}


def parse_expr(text):
    """An infix expression over fields -- "vel[1] * vel[2] / mass + 0.5", "sqrt(fma(a, b, c))"
    -- as the postfix program soax_expr runs: a list of ("load", field, comp),
    ("const", value) and operator names, in Python's operator precedence, left to right.
    A field without a subscript is component 0.  Functions: sqrt, abs, min, max, fma."""
    def walk(node, out):
        if isinstance(node, ast.BinOp) and type(node.op) in _BINOPS:
            walk(node.left, out)
            walk(node.right, out)
            out.append(_BINOPS[type(node.op)])
        elif isinstance(node, ast.UnaryOp) and isinstance(node.op, (ast.USub, ast.UAdd)):
            walk(node.operand, out)
            if isinstance(node.op, ast.USub):
                out.append("neg")
        elif isinstance(node, ast.Call) and isinstance(node.func, ast.Name) and node.func.id in _CALLS:
            name, arity = _CALLS[node.func.id]
            if len(node.args) != arity or node.keywords:
                raise ValueError(f"parse_expr: {node.func.id} takes {arity} arguments")
            for a in node.args:
                walk(a, out)
            out.append(name)
        elif isinstance(node, ast.Subscript) and isinstance(node.value, ast.Name):
            idx = node.slice
            if not (isinstance(idx, ast.Constant) and isinstance(idx.value, int)):
                raise ValueError("parse_expr: a component must be an integer literal")
            out.append(("load", node.value.id, idx.value))
        elif isinstance(node, ast.Name):
            out.append(("load", node.id, 0))
        elif isinstance(node, ast.Constant) and isinstance(node.value, (int, float)) \
                and not isinstance(node.value, bool):
            out.append(("const", float(node.value)))
        else:
            raise ValueError(f"parse_expr: unsupported syntax {ast.dump(node)[:60]}")
        return out
    return walk(ast.parse(text.strip(), mode="eval").body, [])


class SoaxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_LIB = None


def lib():
    """Load libsoax.so (building it in-tree with nvcc if it is missing)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(_abi.LIB_PATH):
            from . import build as _build
            _build.build()
        _LIB = _abi.declare(C.CDLL(_abi.LIB_PATH))
    return _LIB


def _check(rc, what=""):
    if rc != 0:
        msg = lib().soax_last_error().decode(errors="replace")
        raise SoaxError(rc, f"{what}: {msg}" if what else msg)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _ptr3(ts):
    if ts is None:
        return None
    return (C.c_void_p * 3)(*[t.data_ptr() for t in ts])


def _hold(stream, *tensors):
    """Keep device memory this binding allocated for a call alive until the call's work
    on `stream` has run.  The caching allocator frees a tensor against the stream that is
    current when it was allocated; a call launched on another stream can still be using
    it after this function returns, so the tensor is marked as used by that stream too."""
    if stream is None:
        return
    if stream == torch.cuda.current_stream(stream.device):
        return
    for t in tensors:
        if isinstance(t, (list, tuple)):
            _hold(stream, *t)
        elif t is not None and t.is_cuda:
            t.record_stream(stream)


def sync(stream=None):
    """Synchronise the stream and report a device-side error as SoaxError."""
    _check(lib().soax_sync(_stream(stream)), "soax_sync")


@dataclass
class Flow:
    """Parameters of the inertial-particle step (include/soax.h: soax_flow)."""
    A: float = 1.0
    B: float = 1.0
    C: float = 1.0
    tau: float = 0.1
    dt: float = 1e-3
    tau_field: str = None   # name of an f32 x 1 field; tau_i = tau_scale * field[i]
    tau_scale: float = 0.0
    pos: str = "pos"
    vel: str = "vel"
    acc: str = None


@dataclass
class Tune:
    parts_per_thread: int = 4
    block: int = 256
    vec_bits: int = 128
    fuse_steps: int = 0

    def c(self):
        return soax_tune(self.parts_per_thread, self.block, self.vec_bits, self.fuse_steps)


class Particles:
    """n particles of a schema, one torch tensor per (field, component) and buffer set.

    schema: list of (name, dtype in {'i32','i64','u8','f32','f64'}, ncomp, tag).
    shadow: also allocate the second buffer set (needed by sort_by_cell / permute).
    """

    def __init__(self, schema, n, device=None, shadow=True):
        self.schema = [(str(a), str(b), int(c), str(d)) for a, b, c, d in schema]
        self.n = int(n)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self._names = [s[0] for s in self.schema]
        descs = (soax_field_desc * len(self.schema))()
        self._keep = []
        for k, (name, dt, nc, tag) in enumerate(self.schema):
            b = name.encode()
            self._keep.append(b)
            descs[k] = soax_field_desc(b, DTYPES[dt], nc, tag.encode()[:1])
        h = C.c_void_p()
        _check(lib().soax_create(descs, len(self.schema), self.n, C.byref(h)), "soax_create")
        self.h = h
        self.planes = [{}, {}]
        for buf in (0, 1) if shadow else (0,):
            for k, (name, dt, nc, _) in enumerate(self.schema):
                ts = [torch.empty(self.n, dtype=TORCH_DTYPES[dt], device=self.device) for _ in range(nc)]
                for c, t in enumerate(ts):
                    _check(lib().soax_bind(self.h, k, c, buf, _ptr(t) if self.n else None), "soax_bind")
                self.planes[buf][name] = ts

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and _LIB is not None:
            _LIB.soax_destroy(h)
            self.h = None

    # ------------------------------------------------------------------ fields
    def fidx(self, name):
        return self._names.index(name)

    @property
    def current(self):
        b = C.c_int32()
        _check(lib().soax_current(self.h, C.byref(b)))
        return b.value

    def set_current(self, buf):
        _check(lib().soax_set_current(self.h, int(buf)))

    def field(self, name, buf=None):
        """The component tensors of a field in the live (or given) buffer set."""
        return self.planes[self.current if buf is None else buf][name]

    def load(self, arrays):
        """Copy host or device arrays into the live planes: {name: [comp0, comp1, ...]}."""
        for name, comps in arrays.items():
            dst = self.field(name)
            for c, a in enumerate(comps):
                a = torch.as_tensor(a)
                dst[c][: a.shape[0]].copy_(a)

    def copy_plane(self, name, comp, host, to_device, stream=None):
        """soax_copy_plane: one live plane to (to_device=True) or from a host tensor or
        array of the plane's element size and at least n elements, asynchronously on the
        stream (host memory must be pinned for that, and must outlive the copy)."""
        t = torch.as_tensor(host)
        if t.device.type != "cpu" or not t.is_contiguous():
            raise ValueError("copy_plane: host must be a contiguous CPU tensor or array")
        plane = self.field(name)[comp]
        if t.element_size() != plane.element_size() or t.numel() < self.n:
            raise ValueError("copy_plane: host must hold n elements of the plane's size")
        _check(lib().soax_copy_plane(self.h, self.fidx(name), int(comp), C.c_void_p(t.data_ptr()), int(bool(to_device)),
                                     _stream(stream)), "soax_copy_plane")

    def host_planes(self, pinned=True):
        """Host tensors shaped like the planes ({name: [comp0, ...]}, n elements each),
        page-locked by default: the host home of a set that step_host streams."""
        out = {}
        for name, dt, nc, _ in self.schema:
            ts = [torch.empty(self.n, dtype=TORCH_DTYPES[dt]) for _ in range(nc)]
            out[name] = [t.pin_memory() for t in ts] if pinned else ts
        return out

    def step_host(self, host, f: Flow, nsteps, grid, nchunks=0, ws=None, stream=None, up_stream=None,
                  down_stream=None, defer=False):
        """soax_step_host: one sort interval of the set held in the host tensors `host`
        ({name: [comp0, ...]}, contiguous CPU tensors of the planes' element sizes and n
        elements, pinned for overlap): uploaded in nchunks pieces (0: the library's
        default), stepped nsteps fused steps with cell keys on the grid^3 grid, sorted by
        cell, gathered and downloaded back into `host`, all asynchronously: the host
        tensors are final once down_stream has passed the call (synchronise it or the
        device), the device planes once `stream` has.  Copies run on up_stream and
        down_stream (two streams of this object when not given).  defer: leave the
        downloads to the next step_host call (interleaved with its uploads) or to
        step_host_finish; the live planes must not change meanwhile.  Returns the
        permutation (int32 view into ws); with the workspace this object keeps (ws None),
        the next step_host call overwrites it, so it is valid until then."""
        ptrs = []
        for name, dt, nc, _ in self.schema:
            comps = host[name]
            if len(comps) != nc:
                raise ValueError(f"step_host: field {name} needs {nc} host tensors")
            for t in comps:
                if t.device.type != "cpu" or not t.is_contiguous():
                    raise ValueError("step_host: host tensors must be contiguous CPU tensors")
                if t.element_size() != torch.empty(0, dtype=TORCH_DTYPES[dt]).element_size() or t.numel() < self.n:
                    raise ValueError(f"step_host: field {name} needs n elements of its size")
                ptrs.append(t.data_ptr())
        if ws is None:
            # One workspace per grid, kept by this object: the call's keys and permutation
            # live there until its device work has run, which can be long after the call
            # returns (a workspace freed on return could be handed to other work while the
            # call's sort still writes into it).
            # Keyed by the grid and the current size: the workspace grows with n (set_size).
            cache = self.__dict__.setdefault("_host_ws", {})
            if (grid, self.n) not in cache:
                cache[(grid, self.n)] = self.sort_workspace(grid)
            ws = cache[(grid, self.n)]
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        if s != torch.cuda.current_stream(self.device):
            ws.record_stream(s)
        if up_stream is None or down_stream is None:
            if getattr(self, "_copy_streams", None) is None:
                self._copy_streams = (torch.cuda.Stream(self.device), torch.cuda.Stream(self.device))
            up_stream = up_stream or self._copy_streams[0]
            down_stream = down_stream or self._copy_streams[1]
        arr = (C.c_void_p * max(len(ptrs), 1))(*ptrs)
        fl = self.flow(f)
        _check(lib().soax_step_host(self.h, arr, C.byref(fl), int(nsteps), int(grid), int(nchunks), int(bool(defer)),
                                    _ptr(ws), ws.numel(), _stream(stream), _stream(up_stream), _stream(down_stream)),
               "soax_step_host")
        return self.sort_results(grid, ws)[1]

    def step_host_finish(self, down_stream=None):
        """soax_step_host_finish: enqueue the downloads a step_host(defer=True) call left
        (on down_stream, this object's download stream when not given)."""
        if down_stream is None:
            if getattr(self, "_copy_streams", None) is None:
                self._copy_streams = (torch.cuda.Stream(self.device), torch.cuda.Stream(self.device))
            down_stream = self._copy_streams[1]
        _check(lib().soax_step_host_finish(self.h, _stream(down_stream)), "soax_step_host_finish")

    def numpy(self):
        """Live planes (the current size) as numpy arrays (synchronises)."""
        return {name: [t[:self.n].cpu().numpy() for t in self.field(name)] for name in self._names}

    def flow(self, f: Flow):
        return soax_flow(f.A, f.B, f.C, f.tau, f.dt, f.tau_scale,
                         self.fidx(f.tau_field) if f.tau_field else -1, self.fidx(f.pos), self.fidx(f.vel),
                         self.fidx(f.acc) if f.acc else -1)

    # ------------------------------------------------------------------ ops
    def step(self, f: Flow, nsteps=1, stream=None):
        fl = self.flow(f)
        _check(lib().soax_step(self.h, C.byref(fl), int(nsteps), _stream(stream)), "soax_step")

    def step_fused(self, f: Flow, nsteps=1, stream=None, grid=None, keys=None, perm=None):
        """nsteps steps in one pass over the planes (soax_step_fused).  With grid (and
        optionally keys, an int32 tensor of n elements), also the cell keys of the final
        positions (soax_step_fused_keys); returns the keys tensor then.  With perm (int32
        tensor of n elements, e.g. from sort_perm), the permute-gather of every plane by
        perm in the same pass, into the other buffer set (soax_permute_step_fused)."""
        fl = self.flow(f)
        if perm is not None:
            if grid is not None and keys is None:
                keys = torch.empty(max(self.n, 1), dtype=torch.int32, device=self.device)
                _hold(stream, keys)
            _check(lib().soax_permute_step_fused(self.h, _ptr(perm), C.byref(fl), int(nsteps),
                                                 int(grid) if grid is not None else 0, _ptr(keys), _stream(stream)),
                   "soax_permute_step_fused")
            return keys
        if grid is None:
            _check(lib().soax_step_fused(self.h, C.byref(fl), int(nsteps), _stream(stream)), "soax_step_fused")
            return None
        if keys is None:
            keys = torch.empty(max(self.n, 1), dtype=torch.int32, device=self.device)
            _hold(stream, keys)
        _check(lib().soax_step_fused_keys(self.h, C.byref(fl), int(nsteps), int(grid), _ptr(keys), _stream(stream)),
               "soax_step_fused_keys")
        return keys

    def aos_layout(self):
        rb = C.c_int64()
        offs = (C.c_int64 * len(self.schema))()
        _check(lib().soax_aos_layout(self.h, C.byref(rb), offs))
        return rb.value, list(offs)

    def new_aos(self):
        rb, _ = self.aos_layout()
        return torch.empty(self.n * rb, dtype=torch.uint8, device=self.device)

    def to_aos(self, out=None, stream=None):
        if out is None:
            out = self.new_aos()
            _hold(stream, out)
        _check(lib().soax_soa_to_aos(self.h, _ptr(out), _stream(stream)), "soax_soa_to_aos")
        return out

    def from_aos(self, aos, stream=None):
        _check(lib().soax_aos_to_soa(self.h, _ptr(aos), _stream(stream)), "soax_aos_to_soa")

    def step_aos(self, aos, f: Flow, nsteps=1, stream=None):
        fl = self.flow(f)
        _check(lib().soax_step_aos(self.h, _ptr(aos), C.byref(fl), int(nsteps), _stream(stream)), "soax_step_aos")

    def cell_keys(self, grid, pos="pos", out=None, stream=None):
        if out is None:
            out = torch.empty(self.n, dtype=torch.int32, device=self.device)
            _hold(stream, out)
        _check(lib().soax_cell_keys(self.h, self.fidx(pos), int(grid), _ptr(out), _stream(stream)), "soax_cell_keys")
        return out

    def sort_workspace(self, grid):
        b = C.c_size_t()
        _check(lib().soax_sort_workspace_bytes(self.h, int(grid), C.byref(b)))
        return torch.empty(max(b.value, 16), dtype=torch.uint8, device=self.device)

    def sort_by_cell(self, grid, ws=None, stream=None):
        """Cell sort of every field; returns (sorted keys, perm) as int32 views into ws."""
        if ws is None:
            ws = self.sort_workspace(grid)
            _hold(stream, ws)
        _check(lib().soax_sort_by_cell(self.h, int(grid), _ptr(ws), ws.numel(), _stream(stream)), "soax_sort_by_cell")
        return self.sort_results(grid, ws)

    def sort_by_keys(self, grid, keys, ws=None, stream=None):
        """sort_by_cell with the keys given (from step_fused(..., keys=...) or cell_keys):
        no key pass.  Returns (sorted keys, perm) as int32 views into ws."""
        if ws is None:
            ws = self.sort_workspace(grid)
            _hold(stream, ws)
        _check(lib().soax_sort_by_keys(self.h, int(grid), _ptr(keys), _ptr(ws), ws.numel(), _stream(stream)),
               "soax_sort_by_keys")
        return self.sort_results(grid, ws)

    def sort_perm(self, grid, keys, ws=None, stream=None):
        """The stable permutation sorting keys, left in ws (no particle moves); returns
        (None, perm) with perm an int32 view into ws (the sorted keys are not written)."""
        if ws is None:
            ws = self.sort_workspace(grid)
            _hold(stream, ws)
        _check(lib().soax_sort_perm(self.h, int(grid), _ptr(keys), _ptr(ws), ws.numel(), _stream(stream)),
               "soax_sort_perm")
        return None, self.sort_results(grid, ws)[1]

    def sort_results(self, grid, ws):
        k, p = C.c_void_p(), C.c_void_p()
        _check(lib().soax_sort_results(self.h, int(grid), _ptr(ws), ws.numel(), C.byref(k), C.byref(p)))
        base = ws.data_ptr()
        ko, po = (k.value or base) - base, (p.value or base) - base
        kt = ws[ko:ko + 4 * self.n].view(torch.int32)
        pt = ws[po:po + 4 * self.n].view(torch.int32)
        return kt, pt

    def permute(self, perm, stream=None):
        _check(lib().soax_permute(self.h, _ptr(perm), _stream(stream)), "soax_permute")

    @property
    def size(self):
        n = C.c_int64()
        _check(lib().soax_size(self.h, C.byref(n), None, None))
        return n.value

    def set_size(self, n):
        """resize within the capacity given at construction (Listing 5)."""
        _check(lib().soax_set_size(self.h, int(n)), "soax_set_size")
        self.n = int(n)

    def get_element(self, i, stream=None):
        """Particle i as one AoS record (uint8 tensor of the record size, Listing 6)."""
        rb, _ = self.aos_layout()
        rec = torch.empty(max(rb, 16), dtype=torch.uint8, device=self.device)
        _hold(stream, rec)
        _check(lib().soax_get_element(self.h, int(i), _ptr(rec), _stream(stream)), "soax_get_element")
        return rec[:rb]

    def set_element(self, i, rec, stream=None):
        _check(lib().soax_set_element(self.h, int(i), _ptr(rec), _stream(stream)), "soax_set_element")

    def push_back(self, rec, stream=None):
        """Append one particle given as an AoS record (needs spare capacity)."""
        n = self.size
        self.set_size(n + 1)
        self.set_element(n, rec, stream)

    def remove(self, idx, stream=None):
        """Remove the particles at distinct ascending indices (int32 tensor) by overwriting
        each with the last one (Sec. 2)."""
        k = idx.numel()
        b = C.c_size_t()
        _check(lib().soax_remove_workspace_bytes(k, C.byref(b)))
        ws = torch.empty(max(b.value, 16), dtype=torch.uint8, device=self.device)
        _hold(stream, ws)
        _check(lib().soax_remove(self.h, _ptr(idx), k, _ptr(ws), ws.numel(), _stream(stream)), "soax_remove")
        self.n -= k

    def fill(self, value, field=None, stream=None):
        """SetToValue on every array of a field, or of all fields (Listing 7)."""
        _check(lib().soax_fill(self.h, -1 if field is None else self.fidx(field), float(value), _stream(stream)),
               "soax_fill")

    def lincomb(self, dst, terms, constant=0.0, stream=None):
        """dst = constant + sum coef * src in one pass; dst and each src are (field, comp),
        terms a list of ((field, comp), coef).  E.g. Listing 5's
        posArr(0) = velArr(1) - velArr(2): lincomb(("pos", 0), [(("vel", 1), 1), (("vel", 2), -1)])."""
        k = len(terms)
        fs = (C.c_int32 * max(1, k))(*[self.fidx(t[0][0]) for t in terms])
        cs = (C.c_int32 * max(1, k))(*[int(t[0][1]) for t in terms])
        co = (C.c_double * max(1, k))(*[float(t[1]) for t in terms])
        _check(lib().soax_lincomb(self.h, self.fidx(dst[0]), int(dst[1]), k, fs, cs, co, float(constant),
                                  _stream(stream)), "soax_lincomb")

    def expr(self, dst, program, compute="f64", stream=None):
        """soax_expr: dst = program, one pass over the planes involved.  dst is (field,
        comp); program is a postfix list as parse_expr returns it (("load", field, comp),
        ("const", value), operator names) or an infix string for parse_expr; compute is the
        arithmetic type, "f32" or "f64"."""
        prog = parse_expr(program) if isinstance(program, str) else program
        ops = (soax_expr_op * max(1, len(prog)))()
        for j, item in enumerate(prog):
            name = item if isinstance(item, str) else item[0]
            o = ops[j]
            o.op = EXPR_OPS[name]
            if name == "load":
                o.field, o.comp = self.fidx(item[1]), int(item[2])
            elif name == "const":
                o.value = float(item[1])
        _check(lib().soax_expr(self.h, self.fidx(dst[0]), int(dst[1]), ops, len(prog), DTYPES[compute],
                               _stream(stream)), "soax_expr")

    def assign(self, text, compute="f64", stream=None):
        """Listing 5's notation: "pos[0] = vel[1] - vel[2]" (soax_expr of the right-hand side
        into the left-hand plane)."""
        lhs, rhs = text.split("=", 1)
        dst = parse_expr(lhs)
        if len(dst) != 1 or not isinstance(dst[0], tuple) or dst[0][0] != "load":
            raise ValueError("assign: the left-hand side must be one field component")
        self.expr((dst[0][1], dst[0][2]), parse_expr(rhs), compute, stream)

    def euler(self, dt, pos="x", vel="v", per_component=False, stream=None):
        """The paper's Eq. 1 step x += dt*v on f32 x 3 fields (fused, or one launch per
        component as the paper's GPU benchmark)."""
        _check(lib().soax_euler(self.h, self.fidx(pos), self.fidx(vel), float(dt), int(bool(per_component)),
                                _stream(stream)), "soax_euler")

    # ------------------------------------------------------------------ adjoint
    def adjoint_workspace(self, K, ckpt_every):
        b = C.c_size_t()
        _check(lib().soax_adjoint_workspace_bytes(self.h, int(K), int(ckpt_every), C.byref(b)))
        return torch.empty(max(b.value, 16), dtype=torch.uint8, device=self.device)

    def step_checkpointed(self, f: Flow, K, ckpt_every, ws, stream=None):
        fl = self.flow(f)
        _check(lib().soax_step_checkpointed(self.h, C.byref(fl), int(K), int(ckpt_every), _ptr(ws), ws.numel(),
                                            _stream(stream)), "soax_step_checkpointed")

    def step_adjoint(self, f: Flow, K, ckpt_every, ws, xbarK, vbarK=None, stream=None):
        """Returns (xbar0 [3], vbar0 [3], grad[A, B, C, tau]) as f64 tensors."""
        fl = self.flow(f)
        xb0 = [torch.empty(self.n, dtype=torch.float64, device=self.device) for _ in range(3)]
        vb0 = [torch.empty(self.n, dtype=torch.float64, device=self.device) for _ in range(3)]
        grad = torch.empty(4, dtype=torch.float64, device=self.device)
        xk = [t.contiguous() for t in xbarK]
        vk = [t.contiguous() for t in vbarK] if vbarK is not None else None
        _hold(stream, xb0, vb0, grad, xk, vk)
        _check(lib().soax_step_adjoint(self.h, C.byref(fl), int(K), int(ckpt_every), _ptr(ws), ws.numel(),
                                       _ptr3(xk), _ptr3(vk), _ptr3(xb0), _ptr3(vb0), _ptr(grad), _stream(stream)),
               "soax_step_adjoint")
        return xb0, vb0, grad

    def minimage_loss(self, xtgt, ws, want_grad=True, pos="pos", stream=None):
        loss = torch.empty(1, dtype=torch.float64, device=self.device)
        xb = [torch.empty(self.n, dtype=torch.float64, device=self.device) for _ in range(3)] if want_grad else None
        xt = [t.contiguous() for t in xtgt]
        _hold(stream, loss, xb, xt)
        _check(lib().soax_minimage_loss(self.h, self.fidx(pos), _ptr3(xt), _ptr(loss), _ptr3(xb), _ptr(ws),
                                        ws.numel(), _stream(stream)), "soax_minimage_loss")
        return loss, xb


def sort_graph_counts():
    """(built, failed): the cell-sort CUDA graphs this process built, and the builds that
    failed (those sorts launch their kernels on the stream) (soax_sort_graph_counts)."""
    built, failed = C.c_int64(), C.c_int64()
    _check(lib().soax_sort_graph_counts(C.byref(built), C.byref(failed)), "soax_sort_graph_counts")
    return built.value, failed.value


def radix_sort_pairs(keys, vals=None, key_bits=32, want_keys=True, ws=None, stream=None, out=None):
    """Stable LSD radix sort of (u32 key, u32 value); vals None = argsort.  Tensors are
    int32 holding the u32 bit patterns.  Returns (sorted keys or None, sorted values);
    out: a tensor of n int32 to receive the sorted values (else one is allocated)."""
    n = keys.numel()
    b = C.c_size_t()
    _check(lib().soax_radix_workspace_bytes(n, int(key_bits), C.byref(b)))
    if ws is None:
        ws = torch.empty(max(b.value, 16), dtype=torch.uint8, device=keys.device)
        _hold(stream, ws)
    ko = torch.empty_like(keys) if want_keys else None
    vo = torch.empty(n, dtype=torch.int32, device=keys.device) if out is None else out
    _hold(stream, ko, vo if out is None else None)
    _check(lib().soax_radix_sort_pairs(_ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo), n, int(key_bits), _ptr(ws),
                                       ws.numel(), _stream(stream)), "soax_radix_sort_pairs")
    return ko, vo


def euler_aos(rec, n, record_bytes, x_off, v_off, dt, stream=None):
    """Eq. 1 on n AoS records (f32 x[3] at x_off, f32 v[3] at v_off), in place."""
    _check(lib().soax_euler_aos(_ptr(rec), int(n), int(record_bytes), int(x_off), int(v_off), float(dt),
                                _stream(stream)), "soax_euler_aos")


def _handles(parts):
    return (C.c_void_p * len(parts))(*[p.h.value for p in parts])


def _flows(parts, flows):
    arr = (soax_flow * len(parts))()
    for k, (p, f) in enumerate(zip(parts, flows)):
        arr[k] = p.flow(f)
    return arr


def batched_workspace(parts):
    """A fresh workspace for step_batched.  Its address may be one an earlier, freed
    workspace had, so the library is told to forget any plan it recorded there."""
    b = C.c_size_t()
    _check(lib().soax_batched_workspace_bytes(_handles(parts), len(parts), None, C.byref(b)))
    ws = torch.empty(max(b.value, 16), dtype=torch.uint8, device=parts[0].device)
    _check(lib().soax_batched_forget(_ptr(ws)), "soax_batched_forget")
    return ws


def step_batched(parts, flows, nsteps, tune: Tune = None, ws=None, stream=None):
    """Advance every ensemble nsteps steps, one persistent launch per step (bit-identical
    to Particles.step per ensemble) or, with tune.fuse_steps, one launch in total
    (bit-identical to Particles.step_fused per ensemble).  The first call for a new
    (ensembles, tune, ws) uploads a tile plan and synchronises; later identical calls only
    launch."""
    if ws is None:
        ws = batched_workspace(parts)
        _hold(stream, ws)
    t = tune.c() if tune is not None else None
    _check(lib().soax_step_batched(_handles(parts), _flows(parts, flows), len(parts), int(nsteps),
                                   C.byref(t) if t is not None else None, _ptr(ws), ws.numel(), _stream(stream)),
           "soax_step_batched")
    return ws


def _tune_cache_path():
    return os.path.join(os.path.expanduser("~"), ".cache", "soax_b300", "autotune.json")


def _tune_key(parts):
    schema = json.dumps(parts[0].schema)
    total = sum(p.n for p in parts)
    gpu = torch.cuda.get_device_name(parts[0].device)
    return f"{gpu}|{hashlib.sha1(schema.encode()).hexdigest()[:12]}|n2^{total.bit_length()}|e{len(parts)}"


def autotune(parts, flows, nsteps_probe=2, use_cache=True, stream=None, fuse=False):
    """Pick the fastest launch shape for step_batched on these ensembles, for one launch
    per step (fuse=False) or for the fused form (fuse=True: all steps of a call in one
    launch).  Times every candidate on scratch copies (the ensembles are not modified)
    and caches the result in ~/.cache/soax_b300/autotune.json keyed by (GPU, schema,
    size bucket, #ensembles, form)."""
    key = _tune_key(parts) + ("|fused" if fuse else "")
    path = _tune_cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as fh:
                cache = json.load(fh)
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            return Tune(**cache[key])
    scratch = []
    for p in parts:
        q = Particles(p.schema, p.n, device=p.device, shadow=False)
        for name in p._names:
            for c, t in enumerate(p.field(name)):
                q.planes[0][name][c].copy_(t)
        scratch.append(q)
    ws = batched_workspace(scratch)
    out = soax_tune()
    out.fuse_steps = 1 if fuse else 0
    _check(lib().soax_autotune(_handles(scratch), _flows(scratch, flows), len(scratch), int(nsteps_probe), _ptr(ws),
                               ws.numel(), C.byref(out), _stream(stream)), "soax_autotune")
    t = Tune(out.parts_per_thread, out.block, out.vec_bits, out.fuse_steps)
    if use_cache:
        cache[key] = t.__dict__
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path, "w") as fh:
                json.dump(cache, fh, indent=1)
        except OSError:
            pass
    return t


class SoaxRK2(torch.autograd.Function):
    """x_K = RK2^K(x0, v0; A, B, C, tau) with a hand-written adjoint.

    forward(x0 [3, n] f64, v0 [3, n] (f32 values), theta [4] f64 = (A, B, C, tau), dt, K,
    ckpt_every) -> x_K [3, n] f64.  The forward runs soax_step_checkpointed (state saved
    every ckpt_every steps); backward runs soax_step_adjoint, which recomputes each
    segment from its checkpoint.  Gradients flow to x0, v0 and theta."""

    @staticmethod
    def forward(ctx, x0, v0, theta, dt, K, ckpt_every):
        n = x0.shape[1]
        th = [float(t) for t in theta.detach().cpu().tolist()]
        p = Particles([("pos", "f64", 3, "P"), ("vel", "f32", 3, "V")], n, device=x0.device, shadow=False)
        for c in range(3):
            p.planes[0]["pos"][c].copy_(x0[c])
            p.planes[0]["vel"][c].copy_(v0[c])
        f = Flow(A=th[0], B=th[1], C=th[2], tau=th[3], dt=float(dt))
        ws = p.adjoint_workspace(int(K), int(ckpt_every))
        p.step_checkpointed(f, int(K), int(ckpt_every), ws)
        ctx.p, ctx.f, ctx.ws, ctx.K, ctx.C = p, f, ws, int(K), int(ckpt_every)
        ctx.v_dtype = v0.dtype
        return torch.stack([t.clone() for t in p.planes[0]["pos"]])

    @staticmethod
    def backward(ctx, gx):
        gx = gx.to(torch.float64)
        xb0, vb0, grad = ctx.p.step_adjoint(ctx.f, ctx.K, ctx.C, ctx.ws, [gx[c].contiguous() for c in range(3)])
        return torch.stack(xb0), torch.stack(vb0).to(ctx.v_dtype), grad, None, None, None
