"""B300-native geometric-energy fields for haptic assembly (Behandish & Ilies,
"Haptic Assembly Using Skeletal Densities and Fourier Transforms").

A thin Python layer over libhf.so (include/hf.h).  Device memory comes from
torch CUDA tensors, streams from torch streams; every step of the path runs
in the library's sm_103a kernels.  There is no CPU fallback: without the
built library or a CUDA device the calls raise.
"""
import ctypes
import os

import numpy as np

from . import _binding as B
from ._binding import (HF_CKPT_FIELDSET, HF_CKPT_PART, HF_CKPT_SESSION,  # noqa: F401
                       HF_E, HF_F, HF_MOVING, HF_PREC_SPLIT_BF16, HF_PREC_SPLIT_F16, HF_SPECTRAL,
                       HF_STATIONARY, HF_T, HF_TA, HF_TORQUE_C, HF_TORQUE_F64, HFError)

__all__ = ["Context", "Part", "FieldSet", "Batch", "Server", "HFError", "lowpass_query", "lowpass_query_batch",
           "rotation_chunks", "checkpoint_info",
           "resample", "rfft3d", "version"]


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("paper_1711_05017_b300 needs a CUDA device (no CPU fallback)")
    return torch


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, dtype=None):
    torch = _torch()
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def version():
    return B.lib().hf_version().decode()


class Context:
    """hf_ctx: a device and an HBM budget (bytes, 0 = unbounded)."""

    def __init__(self, device=0, hbm_budget_bytes=0):
        _torch()
        h = ctypes.c_void_p()
        B.check(B.lib().hf_ctx_create(int(device), int(hbm_budget_bytes), ctypes.byref(h)))
        self.handle = h
        self.device = device

    def reserved_bytes(self):
        return B.lib().hf_ctx_reserved_bytes(self.handle)

    def resident_queries(self, on=True):
        """hf_ctx_resident_queries: answer FieldSet.query through the resident
        query kernel (no launch per query), or stop it."""
        B.check(B.lib().hf_ctx_resident_queries(self.handle, 1 if on else 0))

    def preload(self):
        """Load every kernel of the builds, torque and queries now (hf_ctx_preload);
        returns the number of kernels in the loaded modules."""
        n = ctypes.c_int()
        B.check(B.lib().hf_ctx_preload(self.handle, ctypes.byref(n)))
        return n.value

    def profile(self, on=True):
        """Bracket every kernel launch of this context with CUDA events."""
        B.check(B.lib().hf_profile_enable(self.handle, 1 if on else 0))

    def profile_read(self, reset=False):
        """{kernel kind: (launches, total device ms)} accumulated so far."""
        L = B.lib()
        n = L.hf_profile_read(self.handle)
        out = {}
        for i in range(n):
            name, cnt, ms = ctypes.c_char_p(), ctypes.c_longlong(), ctypes.c_double()
            B.check(L.hf_profile_entry(self.handle, i, ctypes.byref(name), ctypes.byref(cnt), ctypes.byref(ms)))
            if cnt.value:
                out[name.value.decode()] = (int(cnt.value), float(ms.value))
        if reset:
            L.hf_profile_reset(self.handle)
        return out

    def close(self):
        if self.handle:
            B.lib().hf_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- calls
    def density_build(self, n, pts, sigma, amp=None, out=None, stream=None):
        """hf_density_build: pts (P,3), sigma (P,), amp (P,) or None; float32 CUDA."""
        torch = _torch()
        P = int(sigma.numel())
        if out is None:
            out = torch.empty((n, n, n), dtype=torch.float32, device=sigma.device)
        B.check(B.lib().hf_density_build(self.handle, n, _dev(pts, torch.float32), _dev(sigma, torch.float32),
                                         None if amp is None else _dev(amp, torch.float32), P,
                                         _dev(out, torch.float32), _stream_ptr(stream)))
        return out

    def density_mesh(self, n, V, T, sigma=0.5, gamma_max=0.05, max_depth=8, out=None, aux=None, stream=None):
        """hf_density_mesh: Eq. 2's descriptor of a closed triangle mesh;
        V (nv, 3) float64 and T (nt, 3) int32 CUDA tensors (or numpy arrays,
        copied to the device)."""
        torch = _torch()
        dev = torch.device("cuda", self.device)
        Vt = torch.as_tensor(np.ascontiguousarray(V, dtype=np.float64), device=dev) if not torch.is_tensor(V) else V
        Tt = torch.as_tensor(np.ascontiguousarray(T, dtype=np.int32), device=dev) if not torch.is_tensor(T) else T
        if out is None:
            out = torch.empty((n, n, n), dtype=torch.float32, device=dev)
        B.check(B.lib().hf_density_mesh(self.handle, int(n), _dev(Vt, torch.float64), int(Vt.shape[0]),
                                        _dev(Tt, torch.int32), int(Tt.shape[0]), float(sigma), float(gamma_max),
                                        int(max_depth), _dev(out, torch.float32),
                                        None if aux is None else _dev(aux, torch.float32), _stream_ptr(stream)))
        return out

    def part(self, grid, role, stream=None):
        return Part(self, grid, role, stream)

    def autotune(self, n, cache_path=None):
        """hf_autotune: time the launch shapes for grid size n (or read them
        from cache_path); returns (chunk, pencil, rotations per second)."""
        c, p, r = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        path = None if cache_path is None else str(cache_path).encode()
        B.check(B.lib().hf_autotune(self.handle, int(n), path, ctypes.byref(c), ctypes.byref(p), ctypes.byref(r)))
        return int(c.value), int(p.value), float(r.value)

    def tune_set(self, n, chunk, pencil=False):
        B.check(B.lib().hf_tune_set(self.handle, int(n), int(chunk), 1 if pencil else 0))

    def tune_tiles(self, n, tiles=None):
        """hf_tune_tiles: read, or set to (tile_b, tile_c), the launch shapes
        of passes B and C at grid n."""
        tb, tc = ctypes.c_int(), ctypes.c_int()
        if tiles is not None:
            tb.value, tc.value = int(tiles[0]), int(tiles[1])
        B.check(B.lib().hf_tune_tiles(self.handle, int(n), 1 if tiles is not None else 0, ctypes.byref(tb),
                                      ctypes.byref(tc)))
        return tb.value, tc.value

    def tune_lanes(self, n, lanes=None):
        """hf_tune_lanes: read, or set (1 or 2), the pipelines of a compute at grid n."""
        v = ctypes.c_int(int(lanes) if lanes is not None else 0)
        B.check(B.lib().hf_tune_lanes(self.handle, int(n), 1 if lanes is not None else 0, ctypes.byref(v)))
        return v.value

    def tune_get(self, n):
        c, p, r = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        B.check(B.lib().hf_tune_get(self.handle, int(n), ctypes.byref(c), ctypes.byref(p), ctypes.byref(r)))
        return int(c.value), int(p.value), float(r.value)

    def fieldset(self, n, R, flags=HF_E | HF_F):
        return FieldSet(self, n, R, flags)

    def fields(self, s1, s2, quat, E, Fx=None, Fy=None, Fz=None, scratch=None, stream=None):
        """hf_fields: one rotation into caller buffers."""
        torch = _torch()
        n = s1.n
        if scratch is None:
            nb = B.lib().hf_fields_scratch_bytes(n)
            scratch = torch.empty((nb + 15) // 16 * 4, dtype=torch.float32, device=E.device)
        q = np.ascontiguousarray(quat, dtype=np.float32).reshape(4)
        opt = [None if t is None else _dev(t, torch.float32) for t in (Fx, Fy, Fz)]
        B.check(B.lib().hf_fields(self.handle, s1.handle, s2.handle, B.fptr(q), _dev(E, torch.float32), *opt,
                                  _dev(scratch), _stream_ptr(stream)))
        if stream is not None:
            scratch.record_stream(stream)

    def torque(self, n, quats, E, T, flags=0, stream=None):
        """hf_torque: E (R,N,N,N) -> T (R,3,N,N,N); returns per-rotation status."""
        torch = _torch()
        q = np.ascontiguousarray(quats, dtype=np.float32).reshape(-1, 4)
        R = len(q)
        st = np.zeros(R, dtype=np.int32)
        rc = B.lib().hf_torque(self.handle, n, R, B.fptr(q), _dev(E, torch.float32), _dev(T, torch.float32),
                               int(flags), st.ctypes.data_as(B._ip), _stream_ptr(stream))
        B.check(rc, allow=(B.HF_EINVAL,) if st.any() else ())
        return st


class Part:
    """hf_part: HF_STATIONARY keeps the scaled spectrum, HF_MOVING the grid."""

    def __init__(self, ctx, grid, role, stream=None):
        torch = _torch()
        n = grid.shape[0]
        h = ctypes.c_void_p()
        B.check(B.lib().hf_part_create(ctx.handle, n, _dev(grid, torch.float32), int(role), ctypes.byref(h),
                                       _stream_ptr(stream)))
        self.handle, self.n, self.role, self.ctx = h, n, role, ctx

    def moments(self, stream=None):
        """hf_part_moments: the stationary part's moment spectra for HF_TA
        (analytic torque) field sets."""
        B.check(B.lib().hf_part_moments(self.handle, _stream_ptr(stream)))

    def spectral(self, os=1, stream=None):
        """hf_part_spectral: build the moving part's centred spectrum table
        (padding factor os) for HF_SPECTRAL field sets."""
        B.check(B.lib().hf_part_spectral(self.handle, int(os), _stream_ptr(stream)))

    def save(self, path, stream=None):
        """hf_part_save: the part's state (a moving grid or the stored
        stationary spectrum) to a checkpoint file."""
        B.check(B.lib().hf_part_save(self.handle, os.fsencode(path), _stream_ptr(stream)))

    @classmethod
    def load(cls, ctx, path, stream=None):
        """hf_part_load: a part from a checkpoint file (bitwise the saved state)."""
        h = ctypes.c_void_p()
        B.check(B.lib().hf_part_load(ctx.handle, os.fsencode(path), ctypes.byref(h), _stream_ptr(stream)))
        p = cls.__new__(cls)
        _, n, _, role = checkpoint_info(path)
        p.handle, p.n, p.role, p.ctx = h, n, role, ctx
        return p

    def update(self, grid, stream=None):
        """hf_part_update: re-derive the part from a new grid, in place."""
        torch = _torch()
        B.check(B.lib().hf_part_update(self.handle, _dev(grid, torch.float32), _stream_ptr(stream)))

    def release(self):
        if self.handle:
            B.lib().hf_part_release(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class FieldSet:
    """hf_fieldset: energy, force (and torque) fields for R rotations."""

    def __init__(self, ctx, n, R, flags=HF_E | HF_F):
        h = ctypes.c_void_p()
        B.check(B.lib().hf_fieldset_create(ctx.handle, int(n), int(R), int(flags), ctypes.byref(h)))
        self.handle, self.n, self.R, self.ctx = h, n, R, ctx
        self.flags = B.lib().hf_fieldset_flags(h)

    def compute(self, s1, s2, quats, stream=None, allow_rank_deficient=False):
        q = np.ascontiguousarray(quats, dtype=np.float32).reshape(-1, 4)
        rc = B.lib().hf_fieldset_compute(self.ctx.handle, s1.handle, s2.handle, B.fptr(q), len(q), self.handle,
                                         _stream_ptr(stream))
        return B.check(rc, allow=(B.HF_EINVAL,) if allow_rank_deficient else ())

    def field_ptr(self, rot, field):
        p = ctypes.c_void_p()
        B.check(B.lib().hf_fieldset_field_ptr(self.handle, int(rot), int(field), ctypes.byref(p)))
        return p.value

    def get(self, rot, field, out=None, stream=None):
        torch = _torch()
        if out is None:
            out = torch.empty((self.n,) * 3, dtype=torch.float32, device=f"cuda:{self.ctx.device}")
        B.check(B.lib().hf_fieldset_get(self.handle, int(rot), int(field), _dev(out, torch.float32),
                                        _stream_ptr(stream)))
        return out

    def query(self, t, q, k=4):
        out = np.zeros(7, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32).reshape(3)
        q = np.ascontiguousarray(q, dtype=np.float32).reshape(4)
        B.check(B.lib().hf_query(self.handle, B.fptr(t), B.fptr(q), int(k), B.fptr(out)))
        return out

    def query_batch(self, tq, k=4, out=None, stream=None):
        torch = _torch()
        Q = tq.shape[0]
        if out is None:
            out = torch.empty((Q, 7), dtype=torch.float32, device=tq.device)
        B.check(B.lib().hf_query_batch(self.handle, _dev(tq, torch.float32), int(Q), int(k),
                                       _dev(out, torch.float32), _stream_ptr(stream)))
        return out

    def save(self, path, stream=None):
        """hf_fieldset_save: the computed set (rotations and fields) to a
        checkpoint file."""
        B.check(B.lib().hf_fieldset_save(self.handle, os.fsencode(path), _stream_ptr(stream)))

    @classmethod
    def load(cls, ctx, path, stream=None):
        """hf_fieldset_load: a computed set from a checkpoint file, ready for
        queries (bitwise the saved fields)."""
        h = ctypes.c_void_p()
        B.check(B.lib().hf_fieldset_load(ctx.handle, os.fsencode(path), ctypes.byref(h), _stream_ptr(stream)))
        L = B.lib()
        fs = cls.__new__(cls)
        fs.handle, fs.ctx = h, ctx
        fs.n, fs.R, fs.flags = L.hf_fieldset_n(h), L.hf_fieldset_rotations(h), L.hf_fieldset_flags(h)
        return fs

    def release(self):
        if self.handle:
            B.lib().hf_fieldset_release(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class _BorrowedFieldSet(FieldSet):
    """A field set owned by a Batch: readable, never released from Python."""

    def __init__(self, ctx, handle):
        L = B.lib()
        self.handle, self.ctx = handle, ctx
        self.n, self.R, self.flags = L.hf_fieldset_n(handle), L.hf_fieldset_rotations(handle), L.hf_fieldset_flags(handle)

    def release(self):
        self.handle = None


class Batch:
    """hf_batch: many part pairs (sizes may differ) built by one CUDA graph.
    pairs: [(stationary Part, moving Part)]; R: rotations per pair."""

    def __init__(self, ctx, pairs, R, flags=HF_E | HF_F, slots_per_size=0):
        n = len(pairs)
        S1 = (ctypes.c_void_p * n)(*[p[0].handle.value for p in pairs])
        S2 = (ctypes.c_void_p * n)(*[p[1].handle.value for p in pairs])
        Rs = (ctypes.c_int * n)(*[int(r) for r in R])
        h = ctypes.c_void_p()
        B.check(B.lib().hf_batch_create(ctx.handle, n, S1, S2, Rs, int(flags), int(slots_per_size), ctypes.byref(h)))
        self.handle, self.ctx, self.npairs = h, ctx, n
        self._pairs = list(pairs)

    def set_rotations(self, pair, quats, allow_rank_deficient=False):
        q = np.ascontiguousarray(quats, dtype=np.float32).reshape(-1, 4)
        rc = B.lib().hf_batch_set_rotations(self.handle, int(pair), B.fptr(q))
        return B.check(rc, allow=(B.HF_EINVAL,) if allow_rank_deficient else ())

    def capture(self, lanes=0):
        """Record the whole batch as one graph on `lanes` concurrent branches
        (0: one per slot)."""
        B.check(B.lib().hf_batch_capture(self.handle, int(lanes)))

    def capture_queue(self, chunk=0, spin_limit=0, self_test=0):
        """Record the whole batch as ONE launch of the work-queue kernel
        (hf_batch_capture_queue: E + F, grids 64/96/128)."""
        B.check(B.lib().hf_batch_capture_queue(self.handle, int(chunk), int(spin_limit), int(self_test)))

    def launch(self, stream=None):
        B.check(B.lib().hf_batch_launch(self.handle, _stream_ptr(stream)))

    def status(self, stream=None):
        """hf_batch_status after a one-launch run: (items, runs) of its
        queue; raises HFError(HF_ETIMEOUT) if a bounded wait ran out."""
        it, ru = ctypes.c_int(), ctypes.c_int()
        B.check(B.lib().hf_batch_status(self.handle, _stream_ptr(stream), ctypes.byref(it), ctypes.byref(ru)))
        return it.value, ru.value

    def slots(self):
        return B.lib().hf_batch_slots(self.handle)

    def fieldset(self, pair):
        p = ctypes.c_void_p()
        B.check(B.lib().hf_batch_fieldset(self.handle, int(pair), ctypes.byref(p)))
        return _BorrowedFieldSet(self.ctx, p)

    def release(self):
        if self.handle:
            B.lib().hf_batch_release(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


def lowpass_query(s1, s2, t, q, K=8):
    """hf_lowpass_query: (E, Fx, Fy, Fz, Tx, Ty, Tz) at one pose from spectra
    truncated to |k~| <= K (the moving part needs Part.spectral())."""
    out = np.zeros(7, dtype=np.float32)
    t = np.ascontiguousarray(t, dtype=np.float32).reshape(3)
    q = np.ascontiguousarray(q, dtype=np.float32).reshape(4)
    B.check(B.lib().hf_lowpass_query(s1.handle, s2.handle, int(K), B.fptr(t), B.fptr(q), B.fptr(out)))
    return out


def lowpass_query_batch(s1, s2, tq, K=8, out=None, stream=None):
    """hf_lowpass_query_batch: tq (Q, 7) CUDA float32 -> (Q, 7)."""
    torch = _torch()
    Q = tq.shape[0]
    if out is None:
        out = torch.empty((Q, 7), dtype=torch.float32, device=tq.device)
    B.check(B.lib().hf_lowpass_query_batch(s1.handle, s2.handle, int(K), _dev(tq, torch.float32), int(Q),
                                           _dev(out, torch.float32), _stream_ptr(stream)))
    return out


def resample(rho, R, out=None, stream=None):
    """hf_resample: rho (N,N,N) float32 CUDA, R 3x3 -> rho(R^T x_n)."""
    torch = _torch()
    n = rho.shape[0]
    if out is None:
        out = torch.empty_like(rho)
    r9 = np.ascontiguousarray(R, dtype=np.float32).reshape(9)
    B.check(B.lib().hf_resample(n, _dev(rho, torch.float32), B.fptr(r9), _dev(out, torch.float32),
                                _stream_ptr(stream)))
    return out


def rfft3d(x, out=None, stream=None):
    """hf_rfft3d: (N,N,N) float32 -> (N,N,N/2+1) complex64, natural order."""
    torch = _torch()
    n = x.shape[0]
    if out is None:
        out = torch.empty((n, n, n // 2 + 1), dtype=torch.complex64, device=x.device)
    nb = B.lib().hf_rfft3d_scratch_bytes(n)
    scratch = torch.empty((nb + 15) // 16 * 4, dtype=torch.float32, device=x.device)
    B.check(B.lib().hf_rfft3d(n, _dev(x, torch.float32), _dev(out), _dev(scratch), _stream_ptr(stream)))
    if stream is not None:
        scratch.record_stream(stream)
    return out


def inject_alloc_failure(nth=0):
    """hf_inject_alloc_failure: the library's nth allocation from now on fails
    as out of memory (nth <= 0: off); returns the allocations made so far."""
    c = ctypes.c_longlong()
    B.lib().hf_inject_alloc_failure(int(nth), ctypes.byref(c))
    return c.value


def checkpoint_info(path):
    """hf_checkpoint_info: (kind, N, R, flags) of a checkpoint file (kind
    HF_CKPT_PART / FIELDSET / SESSION; a part's R is 0 and its flags its role)."""
    kind, n, R, fl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_uint()
    B.check(B.lib().hf_checkpoint_info(os.fsencode(path), ctypes.byref(kind), ctypes.byref(n), ctypes.byref(R),
                                       ctypes.byref(fl)))
    return kind.value, n.value, R.value, fl.value


def rotation_chunks(quats, max_build, halo=True):
    """hf_rotation_chunks: split a rotation set into chunks of at most
    max_build rotations per build set (with the 6-nearest torque halo).
    Returns (owner (R,), list of build-set index arrays)."""
    q = np.ascontiguousarray(quats, dtype=np.float32).reshape(-1, 4)
    R = len(q)
    owner = np.zeros(R, dtype=np.int32)
    offs = np.zeros(R + 1, dtype=np.int32)
    build = np.zeros(7 * R, dtype=np.int32)
    C = B.lib().hf_rotation_chunks(B.fptr(q), R, int(max_build), 1 if halo else 0, owner.ctypes.data_as(B._ip),
                                   offs.ctypes.data_as(B._ip), build.ctypes.data_as(B._ip), len(build))
    if C < 1:
        raise HFError(B.HF_EINVAL, "hf_rotation_chunks: invalid arguments")
    return owner, [build[offs[c]:offs[c + 1]].copy() for c in range(C)]


class Server:
    """hf_server: sessions, budgeted continuous batching of field builds, and a
    pool of high-priority query lanes (include/hf.h, serving section)."""

    STATES = {0: "queued", 1: "running", 2: "done", 3: "failed", 4: "superseded"}

    def __init__(self, ctx, max_inflight=4, query_lanes=16):
        h = ctypes.c_void_p()
        B.check(B.lib().hf_server_create(ctx.handle, int(max_inflight), int(query_lanes), ctypes.byref(h)))
        self.handle, self.ctx = h, ctx
        self._parts = {}  # the parts must outlive their sessions: keep them here

    def set_chunk_bytes(self, nbytes):
        """Requests whose field set exceeds nbytes are split into rotation
        chunks (0: never split)."""
        B.check(B.lib().hf_server_set_chunk_bytes(self.handle, int(nbytes)))

    def request_chunks(self, rid, R):
        """(number of chunks, owner chunk of each of the request's R rotations)."""
        c = ctypes.c_int()
        own = np.zeros(R, dtype=np.int32)
        B.check(B.lib().hf_server_request_chunks(self.handle, ctypes.c_int64(rid), ctypes.byref(c),
                                                 own.ctypes.data_as(B._ip)))
        return c.value, own

    def session_save(self, sid, path):
        """hf_server_session_save: the session's published data to a file."""
        B.check(B.lib().hf_server_session_save(self.handle, int(sid), os.fsencode(path)))

    def session_restore(self, sid, path):
        """hf_server_session_restore: a saved session's data as this open
        session's current data."""
        B.check(B.lib().hf_server_session_restore(self.handle, int(sid), os.fsencode(path)))

    def session_counts(self, sid):
        """(queries answered, queries refused as not ready) of a session."""
        a, nr = ctypes.c_int64(), ctypes.c_int64()
        B.check(B.lib().hf_server_session_counts(self.handle, int(sid), ctypes.byref(a), ctypes.byref(nr)))
        return a.value, nr.value

    def trace(self, which):
        """Diagnostic rows since the last read (hf_server_trace): which 0 slow
        queries, 1 slow scheduler calls; an (n, 9) float64 array."""
        buf = np.zeros((4096, 9), dtype=np.float64)
        n = B.lib().hf_server_trace(self.handle, int(which), buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 4096)
        return buf[:n].copy()

    def open(self, s1, s2):
        sid = ctypes.c_int()
        B.check(B.lib().hf_server_session_open(self.handle, s1.handle, s2.handle, ctypes.byref(sid)))
        self._parts[sid.value] = (s1, s2)
        return sid.value

    def close_session(self, sid):
        B.check(B.lib().hf_server_session_close(self.handle, int(sid)))
        self._parts.pop(int(sid), None)

    def submit(self, sid, quats, flags=HF_E | HF_F | HF_T):
        q = np.ascontiguousarray(quats, dtype=np.float32).reshape(-1, 4)
        rid = ctypes.c_int64()
        B.check(B.lib().hf_server_submit(self.handle, int(sid), B.fptr(q), len(q), int(flags), ctypes.byref(rid)))
        return rid.value

    def state(self, rid):
        st, lat = ctypes.c_int(), ctypes.c_double()
        B.check(B.lib().hf_server_request_state(self.handle, ctypes.c_int64(rid), ctypes.byref(st), ctypes.byref(lat)))
        return self.STATES[st.value], lat.value

    def wait(self, rids, timeout=120.0, poll=0.001):
        import time
        t0 = time.time()
        out = {}
        pending = list(rids)
        while pending:
            for r in list(pending):
                st, lat = self.state(r)
                if st in ("done", "failed", "superseded"):
                    out[r] = (st, lat)
                    pending.remove(r)
            if pending:
                if time.time() - t0 > timeout:
                    raise TimeoutError(f"requests {pending} not finished")
                time.sleep(poll)
        return out

    def query(self, sid, t, q, k=4):
        out = np.zeros(7, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32).reshape(3)
        q = np.ascontiguousarray(q, dtype=np.float32).reshape(4)
        B.check(B.lib().hf_server_query(self.handle, int(sid), B.fptr(t), B.fptr(q), int(k), B.fptr(out)))
        return out

    def field_ptr(self, sid, rot, field):
        p = ctypes.c_void_p()
        B.check(B.lib().hf_server_field_ptr(self.handle, int(sid), int(rot), int(field), ctypes.byref(p)))
        return p.value

    def field(self, sid, rot, field, n, stream=None):
        """Copy of a field of the session's current set (torch CUDA tensor)."""
        torch = _torch()
        out = torch.empty((n, n, n), dtype=torch.float32, device=f"cuda:{self.ctx.device}")
        B.check(B.lib().hf_server_field_get(self.handle, int(sid), int(rot), int(field), _dev(out, torch.float32),
                                            _stream_ptr(stream)))
        return out

    def drive_queries(self, sids, poses, rate_hz=1000.0, k=4):
        """Replay poses (nsess, steps, 7) at rate_hz from native threads, one per
        session; blocks.  Returns (answered, not_ready, late)."""
        poses = np.ascontiguousarray(poses, dtype=np.float32)
        s = np.ascontiguousarray(sids, dtype=np.int32)
        a, nr, lt = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        B.check(B.lib().hf_server_drive_queries(self.handle, len(s), s.ctypes.data_as(B._ip), B.fptr(poses),
                                                poses.shape[1], float(rate_hz), int(k), ctypes.byref(a),
                                                ctypes.byref(nr), ctypes.byref(lt)))
        return a.value, nr.value, lt.value

    def query_latencies(self, max_n=1 << 20):
        """Query latencies (us, measured inside the library) since the last read."""
        buf = np.empty(max_n, dtype=np.float32)
        n = B.lib().hf_server_query_latencies(self.handle, B.fptr(buf), int(max_n))
        return buf[:n].copy()

    def log_open(self, path, period_ms=1000):
        """hf_server_log_open: a JSON-lines metrics log appended to `path`
        every period_ms (counters, per-period query and build percentiles)."""
        B.check(B.lib().hf_server_log_open(self.handle, os.fsencode(path), int(period_ms)))

    def log_close(self):
        B.check(B.lib().hf_server_log_close(self.handle))

    def stats(self):
        st = B.ServerStats()
        B.check(B.lib().hf_server_stats_get(self.handle, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in st._fields_}

    def close(self):
        if self.handle:
            B.lib().hf_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

