"""Python binding of the GB300 sampled-space local-energy library (libnqs.so).

Argument marshalling only: every step of the path (staging, FindCoupledPairs,
MatrixElement, ScatterAdd, E^var, adjoint) runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if the library is missing, importing the binding's entry points
raises.

Names follow the paper: ``coupled_pairs`` is FindCoupledPairs, ``local_energy``
returns E_loc^var (Eq. local_energy restricted to the sampled batch),
``variational_energy`` returns E^var (Eq. variational_energy).
"""

import ctypes
import os

import numpy as np
import torch

__all__ = ["NQSError", "load_library", "Hamiltonian", "Batch", "coupled_pairs", "FullCandidates",
           "half_pairs", "local_energy_half", "local_energy_backward_half", "gumbel_topk_level",
           "ar_gumbel_topk", "sr_top", "sr_step",
           "full_candidates", "local_energy_full",
           "local_energy", "variational_energy", "local_energy_backward", "LocalEnergy",
           "evaluate", "BatchedPlan", "SCHEDULES", "PRECISIONS", "library_path",
           "coupled_pairs_async", "ROWS_UNSORTED"]

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "libnqs.so")

SCHEDULES = {"auto": 0, "terms": 1, "batch": 2, "trie": 3}
ROWS_UNSORTED = 0x100   # schedule flag: LoopOverTerms rows left in search order (no row sort)
PRECISIONS = {"fp64": 0, "fp32c": 1}

_c_i64p = ctypes.POINTER(ctypes.c_int64)
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int


class NQSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"nqs error {code}: {msg}")
        self.code = code


_lib = None


def load_library(path: str = None):
    """Load libnqs.so (built by ``paper_2408_07625_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or library_path
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -m paper_2408_07625_gb300.build` (no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    sig = {
        "nqs_ham_load": (_i32, [_i32, _i64, _vp, _vp, _vp, ctypes.POINTER(_vp)]),
        "nqs_ham_free": (_i32, [_vp]),
        "nqs_ham_info": (_i32, [_vp, _c_i64p]),
        "nqs_ham_export": (_i32, [_vp, _vp, _vp, _vp, _vp]),
        "nqs_ham_is_complex": (_i32, [_vp]),
        "nqs_ham_export_im": (_i32, [_vp, _vp]),
        "nqs_stage_bytes": (_i64, [_vp, _i64]),
        "nqs_stage": (_i32, [_vp, _vp, _i64, _vp, _i64, _i32, _vp]),
        "nqs_stage_status": (_i32, [_vp, _vp]),
        "nqs_stage_trie": (_i32, [_vp, _vp, _i64, _vp, _vp]),
        "nqs_count_coupled_pairs": (_i32, [_vp, _vp, _i64, _vp, _i64, _i64, _i32, _vp, _c_i64p, _vp]),
        "nqs_fill_coupled_pairs": (_i32, [_vp, _vp, _i64, _vp, _i64, _i64, _i32, _vp, _vp, _vp, _vp]),
        "nqs_find_coupled_pairs": (_i32, [_vp, _vp, _i64, _vp, _i64, _i64, _i32, _vp, _i64, _vp, _vp, _vp,
                                          _i64, _c_i64p, _vp]),
        "nqs_find_coupled_pairs_async": (_i32, [_vp, _vp, _i64, _vp, _i64, _i64, _i32, _vp, _i64, _vp, _vp,
                                                _vp, _i64, _vp]),
        "nqs_pairs_scratch_bytes": (_i64, [_i64, _i64]),
        "nqs_local_energy": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp, _i64, _i64, _vp, _vp, _vp, _i32,
                                    _vp, _vp, _vp, _vp, _vp]),
        "nqs_variational_energy": (_i32, [_i64, _vp, _vp, _vp, _vp, _vp]),
        "nqs_local_energy_backward": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp, _i64, _i64, _vp, _vp, _vp, _vp,
                                             _vp, _vp, _vp, _vp, _vp, _vp, _vp, _i32, _vp, _vp, _vp]),
        "nqs_batch_plan": (_i32, [_vp, _i32, _i32, _i32, ctypes.POINTER(_vp), _vp]),
        "nqs_batch_run": (_i32, [_vp, _vp]),
        "nqs_batch_status": (_i32, [_vp, ctypes.POINTER(_i32), _vp]),
        "nqs_batch_info": (_i32, [_vp, _i32, _c_i64p]),
        "nqs_batch_tune": (_i32, [_vp, _i32, ctypes.POINTER(ctypes.c_int32)]),
        "nqs_batch_free": (_i32, [_vp]),
        "nqs_evar_combine": (_i32, [_vp, _i32, _vp, _vp]),
        "nqs_evar_combine_host": (_i32, [_vp, _i32, _vp]),
        "nqs_last_error": (ctypes.c_char_p, []),
        "nqs_version": (_i32, []),
        "nqs_search_timing": (_i32, [_i32]),
        "nqs_search_time": (_i32, [ctypes.POINTER(ctypes.c_double), _c_i64p]),
        "nqs_probe_peaks": (_i32, [ctypes.POINTER(ctypes.c_double), _vp]),
        "nqs_candidates_scratch_bytes": (_i64, [_vp, _i64]),
        "nqs_gumbel_scratch_bytes": (_i64, [_i64]),
        "nqs_gumbel_async_max_parents": (_i64, []),
        "nqs_gumbel_topk_level_async": (_i32, [_i32, _i32, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _i64, _vp, _i64,
                                               _vp, _vp, _vp, _vp, _vp]),
        "nqs_sr_scratch_bytes": (_i64, [_i64, _i64]),
        "nqs_sr_top": (_i32, [_i64, _vp, _i64, _vp, _vp, _i64, _vp]),
        "nqs_sr_step": (_i32, [_i32, _i64, _vp, _vp, _vp, _vp, ctypes.c_double, _vp, _vp, _vp, _i64, _vp]),
        "nqs_gumbel_topk_level": (_i32, [_i32, _i32, _i64, _vp, _vp, _vp, _vp, _vp, _i64, _vp, _i64, _vp, _vp, _vp,
                                         _c_i64p, _vp]),
        "nqs_find_pairs_half": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp, _vp, _i64, _c_i64p, _vp]),
        "nqs_find_pairs_part": (_i32, [_vp, _vp, _i64, _vp, _i32, _i32, _vp, _vp, _vp, _i64, _c_i64p, _vp]),
        "nqs_route_scratch_bytes": (_i64, [_i32]),
        "nqs_route_records": (_i32, [_i32, _c_i64p, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _i64, _c_i64p, _vp, _i64,
                                     _vp]),
        "nqs_pairs_from_records": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp, _vp, _i64, _i64, _i64, _vp, _i64, _vp, _vp,
                                          _vp, _i64, _c_i64p, _vp]),
        "nqs_local_energy_half": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _i64, _i32, _vp, _vp, _vp,
                                         _vp, _vp]),
        "nqs_local_energy_backward_half": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp,
                                                  _vp, _vp, _vp, _vp, _vp, _i32, _vp, _vp, _vp]),
        "nqs_full_candidates": (_i32, [_vp, _vp, _i64, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _i64, _c_i64p, _vp]),
        "nqs_local_energy_full": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _i64,
                                         _vp, _vp, _vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc):
    if rc != 0:
        raise NQSError(rc, _lib.nqs_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


_EMPTY = {}


def _pair_ptr(t):
    """Pointer of a pair array; an empty list still passes a valid (unread) buffer."""
    if t is None:
        return None
    if t.numel() == 0:
        key = t.device
        if key not in _EMPTY:
            _EMPTY[key] = torch.zeros(1, dtype=torch.int32, device=t.device)
        return ctypes.c_void_p(_EMPTY[key].data_ptr())
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_u64(U):
    """U as a contiguous int64 CUDA tensor [n, W] holding the uint64 words."""
    if isinstance(U, np.ndarray):
        U = torch.from_numpy(np.ascontiguousarray(U.astype(np.uint64)).view(np.int64))
    if U.dtype not in (torch.int64, torch.uint64):
        raise TypeError("U must hold 64-bit words")
    if U.dtype == torch.uint64:
        U = U.view(torch.int64)
    if U.dim() == 1:
        U = U[:, None]
    if not U.is_cuda:
        U = U.cuda()
    return U.contiguous()


def _f64(t, device):
    if t is None:
        return None
    if isinstance(t, (list, tuple)):
        t = np.asarray(t, dtype=np.float64)
    if isinstance(t, np.ndarray):
        t = torch.from_numpy(np.ascontiguousarray(t, dtype=np.float64))
    return t.to(device=device, dtype=torch.float64).contiguous()


class Hamiltonian:
    """Pauli strings (symplectic x/z masks, real coefficients) grouped by XY on the GPU.

    Follows Sec. "Preparation" (Fig. ham_prep): unique XY patterns, the sets
    P_XY (Eq. xy_to_yz_set) and their term tables.
    """

    def __init__(self, x_mask, z_mask, coef, n_qubits: int):
        lib = load_library()
        x = np.ascontiguousarray(np.asarray(x_mask, dtype=np.uint64))
        z = np.ascontiguousarray(np.asarray(z_mask, dtype=np.uint64))
        c = np.ascontiguousarray(np.asarray(coef, dtype=np.float64).ravel())
        W = max(1, (int(n_qubits) + 63) // 64)
        x = x.reshape(-1, W)
        z = z.reshape(-1, W)
        if not (x.shape[0] == z.shape[0] == c.shape[0]):
            raise ValueError("mask/coef lengths differ")
        h = ctypes.c_void_p()
        _check(lib.nqs_ham_load(int(n_qubits), int(c.shape[0]), x.ctypes.data, z.ctypes.data,
                                c.ctypes.data, ctypes.byref(h)))
        self._h = h
        self.n_qubits = int(n_qubits)
        info = (ctypes.c_int64 * 8)()
        _check(lib.nqs_ham_info(h, info))
        self.info = {"n_qubits": info[0], "n_words": info[1], "n_terms": info[2], "n_xy": info[3],
                     "has_diag": info[4], "max_group": info[5], "n_search": info[6],
                     "heavy_end": info[7]}
        self.n_words = int(info[1])
        self.complex = bool(lib.nqs_ham_is_complex(h))

    @property
    def handle(self):
        return self._h

    def export(self):
        """Host copies of the grouped tables: (xy [n_xy, W], row_ptr, yz [T, W], coef)."""
        W, nxy, T = self.n_words, self.info["n_xy"], self.info["n_terms"]
        xy = np.zeros((nxy, W), np.uint64)
        rp = np.zeros(nxy + 1, np.int64)
        yz = np.zeros((T, W), np.uint64)
        cf = np.zeros(T, np.float64)
        _check(_lib.nqs_ham_export(self._h, xy.ctypes.data, rp.ctypes.data, yz.ctypes.data, cf.ctypes.data))
        return xy, rp, yz, cf

    @classmethod
    def from_instance(cls, inst):
        return cls(inst.x_mask, inst.z_mask, inst.coef, inst.n_qubits)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.nqs_ham_free(self._h)
            self._h = None


class Batch:
    """A staged batch of unique samples U (device) with its workspace."""

    def __init__(self, ham: Hamiltonian, U, check: bool = True, stream=None):
        self.ham = ham
        self.U = _dev_u64(U)
        if self.U.shape[1] != ham.n_words:
            raise ValueError("U word count does not match the Hamiltonian")
        self.n = int(self.U.shape[0])
        self.device = self.U.device
        nbytes = int(_lib.nqs_stage_bytes(ham.handle, self.n))
        if nbytes < 0:
            _check(nbytes)
        self.work = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self._scratch = None          # one-pass search scratch, grown on demand
        self._pair_buf = None         # (pair_j, pair_k) buffers reused between calls
        self._pair_guess = None
        self._async_rp = None         # row_ptr of coupled_pairs_async, reused between calls
        self._packed_buf = None       # packed pair words of coupled_pairs_async, reused between calls
        self._trie = False            # prefix tree of U built since the last staging
        _check(_lib.nqs_stage(ham.handle, _ptr(self.U), self.n, _ptr(self.work), nbytes,
                              1 if check else 0, _stream(stream)))

    def restage(self, U=None, check: bool = False, stream=None):
        """Rebuild the membership structure (for new contents of U, same size)."""
        if U is not None:
            U = _dev_u64(U)
            if tuple(U.shape) != tuple(self.U.shape):
                raise ValueError("restage needs a batch of the same shape")
            self.U = U
        _check(_lib.nqs_stage(self.ham.handle, _ptr(self.U), self.n, _ptr(self.work), self.work.numel(),
                              1 if check else 0, _stream(stream)))
        self._trie = False

    def prefix_tree(self, stream=None):
        """Build the prefix tree of U (Alg. 3) for the trie schedule, once per staging."""
        if not self._trie:
            _check(_lib.nqs_stage_trie(self.ham.handle, _ptr(self.U), self.n, _ptr(self.work), _stream(stream)))
            self._trie = True

    def status(self, stream=None):
        _check(_lib.nqs_stage_status(_ptr(self.work), _stream(stream)))


def count_pairs(batch: Batch, row_begin=0, row_end=None, schedule="terms", stream=None):
    row_end = batch.n if row_end is None else int(row_end)
    if schedule == "trie":
        batch.prefix_tree(stream)
    row_ptr = torch.empty(row_end - row_begin + 1, dtype=torch.int64, device=batch.device)
    n = ctypes.c_int64()
    _check(_lib.nqs_count_coupled_pairs(batch.ham.handle, _ptr(batch.U), batch.n, _ptr(batch.work),
                                        int(row_begin), row_end, SCHEDULES[schedule], _ptr(row_ptr),
                                        ctypes.byref(n), _stream(stream)))
    return row_ptr, int(n.value)


def fill_pairs(batch: Batch, row_ptr, n_pairs, row_begin=0, row_end=None, schedule="terms", stream=None,
               sort_rows=True):
    row_end = batch.n if row_end is None else int(row_end)
    if schedule == "trie":
        batch.prefix_tree(stream)
    pj = torch.empty(max(n_pairs, 1), dtype=torch.int32, device=batch.device)
    pk = torch.empty(max(n_pairs, 1), dtype=torch.int32, device=batch.device)
    sched = SCHEDULES[schedule] | (0 if sort_rows else ROWS_UNSORTED)
    _check(_lib.nqs_fill_coupled_pairs(batch.ham.handle, _ptr(batch.U), batch.n, _ptr(batch.work),
                                       int(row_begin), row_end, sched, _ptr(row_ptr),
                                       _pair_ptr(pj), _pair_ptr(pk), _stream(stream)))
    return pj[:n_pairs], pk[:n_pairs]


def _grow(batch, rows, max_pairs):
    nbytes = int(_lib.nqs_pairs_scratch_bytes(rows, max_pairs))
    if batch._scratch is None or batch._scratch.numel() < nbytes:
        batch._scratch = torch.empty(nbytes, dtype=torch.uint8, device=batch.device)
    if batch._pair_buf is None or batch._pair_buf[0].numel() < max_pairs:
        batch._pair_buf = (torch.empty(max(max_pairs, 1), dtype=torch.int32, device=batch.device),
                           torch.empty(max(max_pairs, 1), dtype=torch.int32, device=batch.device))


def coupled_pairs(batch: Batch, row_begin=0, row_end=None, schedule="terms", one_pass=True,
                  reuse=False, stream=None, sort_rows=True):
    """FindCoupledPairs over rows [row_begin, row_end): CSR (row_ptr, j, k) as CUDA tensors.

    ``j`` and ``k`` are int32 tensors holding uint32 column and pattern indices.
    Each row holds its diagonal pair first, then the rest by ascending column;
    with ``sort_rows=False`` (LoopOverTerms) the rest stay in the order the
    search placed them (same pairs, no row sort): enough for ``local_energy``
    and ``local_energy_backward``, whose row sums do not depend on the order.
    With ``one_pass`` the search runs once, writing into a scratch kept on the
    batch (grown and retried through the fill pass when too small).  With
    ``reuse`` the returned pair tensors are views of buffers that the next
    call on this batch overwrites.
    """
    row_end = batch.n if row_end is None else int(row_end)
    rows = row_end - int(row_begin)
    if schedule == "trie":
        batch.prefix_tree(stream)
    if not one_pass:
        row_ptr, n = count_pairs(batch, row_begin, row_end, schedule, stream)
        pj, pk = fill_pairs(batch, row_ptr, n, row_begin, row_end, schedule, stream, sort_rows)
        return row_ptr, pj, pk
    flag = 0 if sort_rows else ROWS_UNSORTED
    guess = batch._pair_guess or max(256 * rows, 1024)
    _grow(batch, rows, guess)
    row_ptr = torch.empty(rows + 1, dtype=torch.int64, device=batch.device)
    n = ctypes.c_int64()
    pj, pk = batch._pair_buf
    rc = _lib.nqs_find_coupled_pairs(batch.ham.handle, _ptr(batch.U), batch.n, _ptr(batch.work),
                                     int(row_begin), row_end, SCHEDULES[schedule] | flag, _ptr(batch._scratch),
                                     batch._scratch.numel(), _ptr(row_ptr), _ptr(pj), _ptr(pk),
                                     pj.numel(), ctypes.byref(n), _stream(stream))
    total = int(n.value)
    batch._pair_guess = max(guess, int(total * 1.15) + 1024)
    if rc == -4:  # scratch or buffers too small: row_ptr is valid, complete with the fill pass
        _grow(batch, rows, batch._pair_guess)
        pj, pk = batch._pair_buf
        _check(_lib.nqs_fill_coupled_pairs(batch.ham.handle, _ptr(batch.U), batch.n, _ptr(batch.work),
                                           int(row_begin), row_end, SCHEDULES[schedule] | flag, _ptr(row_ptr),
                                           _pair_ptr(pj), _pair_ptr(pk), _stream(stream)))
    else:
        _check(rc)
    if reuse:
        return row_ptr, pj[:total], pk[:total]
    return row_ptr, pj[:total].clone(), pk[:total].clone()


def coupled_pairs_async(batch: Batch, capacity, row_begin=0, row_end=None, schedule="terms",
                        sort_rows=True, packed=False, stream=None):
    """FindCoupledPairs with no host wait: (row_ptr, j, k) with j, k of length ``capacity``.

    With ``packed`` (LoopOverTerms, ``sort_rows=False``) the pairs come as one
    int64 tensor of (column << 32 | pattern) words and ``k`` is None; that is
    the form ``local_energy`` and ``local_energy_backward`` read without a
    split pass.

    The pair total stays on the device (``row_ptr[-1]``); the buffers are kept
    on the batch and reused by the next call.  If the pairs do not fit,
    nothing is written and the batch's status (``Batch.status()``) reports
    NQS_ERR_CAPACITY; later ``local_energy`` / ``local_energy_backward`` calls
    on the batch skip their rows until a call fits.
    """
    row_end = batch.n if row_end is None else int(row_end)
    rows = row_end - int(row_begin)
    capacity = int(capacity)
    if schedule == "trie":
        batch.prefix_tree(stream)
    _grow(batch, rows, max(capacity, 1))
    if batch._async_rp is None or batch._async_rp.numel() != rows + 1:
        batch._async_rp = torch.empty(rows + 1, dtype=torch.int64, device=batch.device)
    row_ptr = batch._async_rp
    pj, pk = batch._pair_buf
    if packed:
        if batch._packed_buf is None or batch._packed_buf.numel() < max(capacity, 1):
            batch._packed_buf = torch.empty(max(capacity, 1), dtype=torch.int64, device=batch.device)
        pj, pk = batch._packed_buf, None
    flag = 0 if sort_rows else ROWS_UNSORTED
    scratch = batch._scratch if schedule in ("terms", "auto") else None
    _check(_lib.nqs_find_coupled_pairs_async(
        batch.ham.handle, _ptr(batch.U), batch.n, _ptr(batch.work), int(row_begin), row_end,
        SCHEDULES[schedule] | flag, _ptr(scratch), 0 if scratch is None else scratch.numel(),
        _ptr(row_ptr), _ptr(pj), _ptr(pk), capacity, _stream(stream)))
    return row_ptr, pj[:capacity], (None if pk is None else pk[:capacity])


def search_timing(on: bool):
    """Bracket every LoopOverTerms search launch with CUDA events (benchmarks)."""
    _check(load_library().nqs_search_timing(1 if on else 0))


def search_time():
    """(summed kernel ms, launches) of the search launches timed since the last call."""
    t = ctypes.c_double()
    n = ctypes.c_int64()
    _check(load_library().nqs_search_time(ctypes.byref(t), ctypes.byref(n)))
    return t.value, int(n.value)


def probe_peaks(stream=None):
    """Measured (integer lane-ops/s of the probe ALU mix, filter-loop probes/s) of this GPU."""
    out = (ctypes.c_double * 2)()
    _check(load_library().nqs_probe_peaks(out, _stream(stream)))
    return float(out[0]), float(out[1])


def pair_h_buffer(n_pairs, precision="fp32c", device="cuda", complex_h=False):
    """A tensor that holds one matrix element per pair (``hpair`` of local_energy);
    both parts of it for a complex Hamiltonian."""
    m = 2 if complex_h else 1
    if precision == "fp64":
        return torch.empty((max(int(n_pairs), 1), m), dtype=torch.float64, device=device).squeeze(1)
    return torch.empty((max(int(n_pairs), 1), 2 * m), dtype=torch.float32, device=device)


def _check_hpair(hpair, n_pairs, precision, complex_h=False):
    if hpair is None:
        return None
    m = 2 if complex_h else 1
    want = (torch.float64, m) if precision == "fp64" else (torch.float32, 2 * m)
    if hpair.dtype != want[0] or hpair.numel() < want[1] * n_pairs or not hpair.is_contiguous():
        raise ValueError("hpair does not match the pair count or precision")
    return hpair


def local_energy(batch: Batch, logpsi_re, logpsi_im=None, pairs=None, precision="fp32c",
                 row_begin=0, row_end=None, out=None, hpair=None, stream=None):
    """E_loc^var for rows [row_begin, row_end) from their CSR pairs.

    Returns (eloc_re, eloc_im or None, hdiag), full-length tensors of which the
    rows in range are written.  ``hpair`` (from ``pair_h_buffer``) receives
    each pair's matrix element for the adjoint.
    """
    row_end = batch.n if row_end is None else int(row_end)
    dev = batch.device
    a = _f64(logpsi_re, dev)
    b = _f64(logpsi_im, dev)
    if pairs is None:
        pairs = coupled_pairs(batch, row_begin, row_end, stream=stream)
    rp, pj, pk = pairs
    cplx = b is not None or batch.ham.complex
    if out is None:
        er = torch.zeros(batch.n, dtype=torch.float64, device=dev)
        ei = torch.zeros(batch.n, dtype=torch.float64, device=dev) if cplx else None
        hd = torch.zeros(batch.n, dtype=torch.float64, device=dev)
    else:
        er, ei, hd = out
    hpair = _check_hpair(hpair, int(pj.numel()), precision, batch.ham.complex)
    _check(_lib.nqs_local_energy(batch.ham.handle, _ptr(batch.U), batch.n, _ptr(batch.work), _ptr(a), _ptr(b),
                                 int(row_begin), row_end, _ptr(rp), _pair_ptr(pj), _pair_ptr(pk),
                                 PRECISIONS[precision], _ptr(er), _ptr(ei), _ptr(hd), _ptr(hpair),
                                 _stream(stream)))
    return er, ei, hd


def variational_energy(batch: Batch, logpsi_re, eloc_re, out=None, stream=None):
    """E^var (Eq. variational_energy) as a device tensor [E, max Re log psi, sum of weights]."""
    a = _f64(logpsi_re, eloc_re.device)
    if out is None:
        out = torch.empty(3, dtype=torch.float64, device=eloc_re.device)
    _check(_lib.nqs_variational_energy(int(a.shape[0]), _ptr(a), _ptr(eloc_re), _ptr(batch.work), _ptr(out),
                                       _stream(stream)))
    return out


def local_energy_backward(batch: Batch, logpsi_re, logpsi_im, eloc_re, eloc_im, hdiag, evar,
                          g_eloc_re=None, g_eloc_im=None, g_evar=None, pairs=None, precision="fp32c",
                          row_begin=0, row_end=None, out=None, hpair=None, stream=None):
    """Gradient of sum g_re Re E_loc + g_im Im E_loc + g_E E^var w.r.t. (Re, Im) log psi.

    ``hpair``: the matrix elements local_energy stored for the same pairs (or
    None to recompute them; the result is the same).
    """
    row_end = batch.n if row_end is None else int(row_end)
    dev = batch.device
    a = _f64(logpsi_re, dev)
    b = _f64(logpsi_im, dev)
    if (g_eloc_re is not None or g_eloc_im is not None) and pairs is None:
        pairs = coupled_pairs(batch, row_begin, row_end, stream=stream)
    rp, pj, pk = pairs if pairs is not None else (None, None, None)
    if out is None:
        gr = torch.zeros(batch.n, dtype=torch.float64, device=dev)
        gi = torch.zeros(batch.n, dtype=torch.float64, device=dev) if b is not None else None
    else:
        gr, gi = out
    # converted arguments are held in locals until the call has been enqueued: a temporary
    # freed after its pointer was taken would let the next conversion reuse its memory
    up_re, up_im, up_e = _f64(g_eloc_re, dev), _f64(g_eloc_im, dev), _f64(g_evar, dev)
    _check(_lib.nqs_local_energy_backward(
        batch.ham.handle, _ptr(batch.U), batch.n, _ptr(batch.work), _ptr(a), _ptr(b), int(row_begin), row_end,
        _ptr(rp), _pair_ptr(pj), _pair_ptr(pk),
        _ptr(_check_hpair(hpair, int(pj.numel()), precision, batch.ham.complex) if pj is not None else None),
        _ptr(eloc_re), _ptr(eloc_im), _ptr(hdiag), _ptr(evar),
        _ptr(up_re), _ptr(up_im), _ptr(up_e),
        PRECISIONS[precision], _ptr(gr), _ptr(gi), _stream(stream)))
    return gr, gi


def _row_chunks(row_ptr_host, max_pairs):
    """Split rows into contiguous ranges holding at most max_pairs pairs each."""
    n = len(row_ptr_host) - 1
    chunks, start = [], 0
    while start < n:
        limit = row_ptr_host[start] + max_pairs
        end = int(np.searchsorted(row_ptr_host, limit, side="right")) - 1
        end = max(end, start + 1)
        end = min(end, n)
        chunks.append((start, end))
        start = end
    return chunks


def evaluate(batch: Batch, logpsi_re, logpsi_im=None, precision="fp32c", schedule="terms",
             max_pairs=None, keep_pairs=True, keep_h=False, stream=None):
    """Whole forward path: FindCoupledPairs, E_loc^var, E^var.

    Without ``max_pairs`` the search runs once (one-pass mode).  With it, rows
    are split into contiguous chunks holding at most ``max_pairs`` pairs each,
    and each chunk's pairs are listed, consumed and dropped in turn.
    Returns dict(eloc_re, eloc_im, hdiag, evar, n_pairs, pairs or None, chunks,
    hpair).  With ``keep_h`` (and a single chunk) ``hpair`` holds each pair's
    matrix element for the adjoint.
    """
    dev = batch.device
    a = _f64(logpsi_re, dev)
    b = _f64(logpsi_im, dev)
    er = torch.zeros(batch.n, dtype=torch.float64, device=dev)
    ei = torch.zeros(batch.n, dtype=torch.float64, device=dev) if (b is not None or batch.ham.complex) else None
    hd = torch.zeros(batch.n, dtype=torch.float64, device=dev)
    rp_host = None
    kept = None
    hpair = None
    if max_pairs is None:
        pairs = coupled_pairs(batch, 0, batch.n, schedule, reuse=not keep_pairs, stream=stream,
                              sort_rows=keep_pairs)
        row_ptr, total, chunks = pairs[0], int(pairs[1].numel()), [(0, batch.n)]
        if keep_h:
            hpair = pair_h_buffer(total, precision, dev, batch.ham.complex)
        local_energy(batch, a, b, pairs, precision, 0, batch.n, (er, ei, hd), hpair=hpair, stream=stream)
        kept = pairs if keep_pairs else None
    else:
        row_ptr, total = count_pairs(batch, 0, batch.n, schedule, stream)
        rp_host = row_ptr.cpu().numpy()
        chunks = _row_chunks(rp_host, int(max_pairs)) if total > max_pairs else [(0, batch.n)]
        for (r0, r1) in chunks:
            rp = row_ptr[r0:r1 + 1]
            pj, pk = fill_pairs(batch, rp, int(rp_host[r1] - rp_host[r0]), r0, r1, schedule, stream,
                                sort_rows=keep_pairs and len(chunks) == 1)
            local_energy(batch, a, b, (rp, pj, pk), precision, r0, r1, (er, ei, hd), stream=stream)
            if len(chunks) == 1 and keep_pairs:
                kept = (rp, pj, pk)
    evar = variational_energy(batch, a, er, stream=stream)
    return {"eloc_re": er, "eloc_im": ei, "hdiag": hd, "evar": evar, "n_pairs": total,
            "pairs": kept, "chunks": chunks, "row_ptr": row_ptr, "row_ptr_host": rp_host,
            "schedule": schedule, "hpair": hpair if kept is not None else None}


class LocalEnergy(torch.autograd.Function):
    """(E_loc^var re, E_loc^var im, E^var) as a differentiable function of log psi.

    ``forward(ctx, batch, logpsi_re, logpsi_im, precision, max_pairs)``; pass
    ``logpsi_im=None`` for real amplitudes (then the second output is zeros).
    The pair list is kept for the backward pass when it fits under
    ``max_pairs``; otherwise the backward pass recomputes it row chunk by row
    chunk.
    """

    @staticmethod
    def forward(ctx, batch, logpsi_re, logpsi_im, precision="fp32c", max_pairs=None):
        res = evaluate(batch, logpsi_re.detach(), None if logpsi_im is None else logpsi_im.detach(),
                       precision, "terms", max_pairs, keep_pairs=True, keep_h=max_pairs is None)
        ctx.batch, ctx.precision, ctx.max_pairs = batch, precision, max_pairs
        ctx.res = res
        ctx.cplx = logpsi_im is not None
        ctx.cplx_out = ctx.cplx or batch.ham.complex   # Im E_loc is not zero
        ctx.save_for_backward(logpsi_re, logpsi_im if logpsi_im is not None else logpsi_re)
        ei = res["eloc_im"] if res["eloc_im"] is not None else torch.zeros_like(res["eloc_re"])
        return res["eloc_re"], ei, res["evar"][0]

    @staticmethod
    def backward(ctx, g_er, g_ei, g_e):
        lre, lim = ctx.saved_tensors
        lim = lim if ctx.cplx else None
        res, batch = ctx.res, ctx.batch
        g_er = None if g_er is None else g_er.contiguous()
        g_ei = None if (g_ei is None or not ctx.cplx_out) else g_ei.contiguous()
        g_e = None if g_e is None else g_e.reshape(1).to(torch.float64).contiguous()
        need_pairs = g_er is not None or g_ei is not None
        if not need_pairs or res["pairs"] is not None:
            gr, gi = local_energy_backward(batch, lre, lim, res["eloc_re"], res["eloc_im"], res["hdiag"],
                                           res["evar"], g_er, g_ei, g_e, res["pairs"], ctx.precision,
                                           hpair=res["hpair"] if need_pairs else None)
        else:
            gr = torch.zeros(batch.n, dtype=torch.float64, device=batch.device)
            gi = torch.zeros(batch.n, dtype=torch.float64, device=batch.device) if ctx.cplx else None
            row_ptr, rp_host = res["row_ptr"], res["row_ptr_host"]
            if rp_host is None:
                rp_host = row_ptr.cpu().numpy()
            for (r0, r1) in res["chunks"]:
                rp = row_ptr[r0:r1 + 1]
                npairs = int(rp_host[r1] - rp_host[r0])
                pj, pk = fill_pairs(batch, rp, npairs, r0, r1, res["schedule"], sort_rows=False)
                local_energy_backward(batch, lre, lim, res["eloc_re"], res["eloc_im"], res["hdiag"],
                                      res["evar"], g_er, g_ei, g_e, (rp, pj, pk), ctx.precision,
                                      r0, r1, (gr, gi))
        return None, gr, gi, None, None


def half_pairs(batch: Batch, stream=None, part=0, n_parts=1):
    """Each unordered coupled pair {x_i, x_j} once as a record (i, j, k) (nqs_find_pairs_half).

    Returns (rec_i, rec_j, rec_k, n_slots): int32 tensors holding uint32 values,
    slots [0, n_slots) of which are in use; an unused slot has i = 0xFFFFFFFF.
    With ``n_parts`` > 1 only slice ``part`` of the search's work items is
    searched (nqs_find_pairs_part).  The buffers are kept on the batch and
    reused by the next call.
    """
    lib = load_library()
    n = ctypes.c_int64()
    cap = getattr(batch, "_half_cap", None) or max(128 * batch.n // max(1, n_parts), 1 << 16)
    for _ in range(3):
        buf = getattr(batch, "_half_buf", None)
        if buf is None or buf[0].numel() < cap:
            buf = tuple(torch.empty(cap, dtype=torch.int32, device=batch.device) for _ in range(3))
            batch._half_buf = buf
        rc = lib.nqs_find_pairs_part(batch.ham.handle, _ptr(batch.U), batch.n, _ptr(batch.work), int(part),
                                     int(n_parts), _ptr(buf[0]), _ptr(buf[1]), _ptr(buf[2]), buf[0].numel(),
                                     ctypes.byref(n), _stream(stream))
        if rc == -4:
            cap = int(n.value * 1.1) + 4096
            batch._half_cap = cap
            continue
        _check(rc)
        break
    else:
        _check(rc)
    k = int(n.value)
    return buf[0][:k], buf[1][:k], buf[2][:k], k


def route_records(records, bounds, stream=None):
    """Copies of half-stored records grouped by the part owning each endpoint row (nqs_route_records).

    ``records``: (rec_i, rec_j, rec_k, n_slots) as from ``half_pairs``;
    ``bounds``: the n_parts + 1 row bounds of the parts.  Returns
    (out_i, out_j, out_k, counts): int32 device tensors grouped by part and the
    host list of each part's number of records.
    """
    lib = load_library()
    ri, rj, rk, ns = records
    b = np.ascontiguousarray(np.asarray(bounds, dtype=np.int64))
    n_parts = len(b) - 1
    dev = ri.device
    nbytes = int(lib.nqs_route_scratch_bytes(n_parts))
    _check(nbytes if nbytes < 0 else 0)
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    counts = (ctypes.c_int64 * n_parts)()
    cap = 2 * max(int(ns), 1)
    out = tuple(torch.empty(cap, dtype=torch.int32, device=dev) for _ in range(3))
    _check(lib.nqs_route_records(n_parts, b.ctypes.data_as(_c_i64p), _pair_ptr(ri), _pair_ptr(rj), _pair_ptr(rk),
                                 int(ns), _ptr(out[0]), _ptr(out[1]), _ptr(out[2]), cap, counts, _ptr(scratch),
                                 nbytes, _stream(stream)))
    c = [int(v) for v in counts]
    tot = sum(c)
    return out[0][:tot], out[1][:tot], out[2][:tot], c


def pairs_from_records(batch: Batch, rec_i, rec_j, rec_k, row_begin, row_end, stream=None):
    """CSR (row_ptr, j, k) of rows [row_begin, row_end) from records naming every pair of those rows
    (nqs_pairs_from_records); the same lists as ``coupled_pairs`` over that range."""
    lib = load_library()
    rows = int(row_end) - int(row_begin)
    dev = batch.device
    n_rec = int(rec_i.numel())
    rp = torch.empty(rows + 1, dtype=torch.int64, device=dev)
    n = ctypes.c_int64()
    cap = max(2 * n_rec + rows, 1)
    for _ in range(2):
        pj = torch.empty(cap, dtype=torch.int32, device=dev)
        pk = torch.empty(cap, dtype=torch.int32, device=dev)
        scratch = torch.empty(256 + 8 * cap, dtype=torch.uint8, device=dev)
        rc = lib.nqs_pairs_from_records(batch.ham.handle, _ptr(batch.U), batch.n, _ptr(batch.work), _pair_ptr(rec_i),
                                        _pair_ptr(rec_j), _pair_ptr(rec_k), n_rec, int(row_begin), int(row_end),
                                        _ptr(scratch), scratch.numel(), _ptr(rp), _ptr(pj), _ptr(pk), cap,
                                        ctypes.byref(n), _stream(stream))
        if rc == -4:
            cap = int(n.value) + 1
            continue
        _check(rc)
        break
    else:
        _check(rc)
    k = int(n.value)
    return rp, pj[:k], pk[:k]


def half_h_buffer(n_slots, precision="fp32c", device="cuda", complex_h=False):
    """Per-record matrix elements of the half-stored path (same layout as pair_h_buffer)."""
    return pair_h_buffer(n_slots, precision, device, complex_h)


def local_energy_half(batch: Batch, logpsi_re, logpsi_im, half, precision="fp32c", out=None, hrec=None,
                      stream=None):
    """E_loc^var from half-stored records (symmetric scatter): (eloc_re, eloc_im or None, hdiag)."""
    dev = batch.device
    a, b = _f64(logpsi_re, dev), _f64(logpsi_im, dev)
    ri, rj, rk, ns = half
    cplx = b is not None or batch.ham.complex
    if out is None:
        er = torch.empty(batch.n, dtype=torch.float64, device=dev)
        ei = torch.empty(batch.n, dtype=torch.float64, device=dev) if cplx else None
        hd = torch.empty(batch.n, dtype=torch.float64, device=dev)
    else:
        er, ei, hd = out
    _check(_lib.nqs_local_energy_half(batch.ham.handle, _ptr(batch.U), batch.n, _ptr(batch.work), _ptr(a), _ptr(b),
                                      _pair_ptr(ri), _pair_ptr(rj), _pair_ptr(rk), ns, PRECISIONS[precision],
                                      _ptr(er), _ptr(ei), _ptr(hd),
                                      _ptr(_check_hpair(hrec, ns, precision, batch.ham.complex)), _stream(stream)))
    return er, ei, hd


def local_energy_backward_half(batch: Batch, logpsi_re, logpsi_im, eloc_re, eloc_im, hdiag, evar, g_eloc_re=None,
                               g_eloc_im=None, g_evar=None, half=None, precision="fp32c", hrec=None, out=None,
                               stream=None):
    """Adjoint over half-stored records (see local_energy_backward): (grad_re, grad_im or None)."""
    dev = batch.device
    a, b = _f64(logpsi_re, dev), _f64(logpsi_im, dev)
    ri, rj, rk, ns = half if half is not None else (None, None, None, 0)
    if out is None:
        gr = torch.empty(batch.n, dtype=torch.float64, device=dev)
        gi = torch.empty(batch.n, dtype=torch.float64, device=dev) if b is not None else None
    else:
        gr, gi = out
    up_re, up_im, up_e = _f64(g_eloc_re, dev), _f64(g_eloc_im, dev), _f64(g_evar, dev)   # held until enqueued
    _check(_lib.nqs_local_energy_backward_half(
        batch.ham.handle, _ptr(batch.U), batch.n, _ptr(batch.work), _ptr(a), _ptr(b), _pair_ptr(ri), _pair_ptr(rj),
        _pair_ptr(rk), ns, _ptr(_check_hpair(hrec, ns, precision, batch.ham.complex)), _ptr(eloc_re), _ptr(eloc_im),
        _ptr(hdiag), _ptr(evar), _ptr(up_re), _ptr(up_im), _ptr(up_e),
        PRECISIONS[precision], _ptr(gr), _ptr(gi), _stream(stream)))
    return gr, gi


_GUMBEL_BYTES = {}   # scratch bytes of nqs_gumbel_topk_level by parent count


def gumbel_topk_level(n_qubits, level, parent_x, parent_l, parent_lt, cond_logp, gumbel, K, device="cuda",
                      stream=None, out=None, scratch=None):
    """One qubit of Alg. 1 (ARGumbelTopK) on the GPU: (child_x [m, W] int64, child_l, child_lt).

    out: optional (child_x, child_l, child_lt) device tensors with room for
    min(K, 2 n_parents) vectors; scratch: optional uint8 device tensor of at
    least nqs_gumbel_scratch_bytes(n_parents) bytes (the returned tensors are
    then views of ``out``)."""
    lib = _lib if _lib is not None else load_library()
    W = (int(n_qubits) + 63) // 64

    def dev(t):   # device FP64, flat; tensors already so pass through untouched
        if torch.is_tensor(t) and t.dtype == torch.float64 and t.is_cuda and t.is_contiguous():
            return t.view(-1)
        if not torch.is_tensor(t):
            t = np.asarray(t, dtype=np.float64).reshape(-1)
        return _f64(t, device).view(-1)

    pl, plt, lp, g = dev(parent_l), dev(parent_lt), dev(cond_logp), dev(gumbel)
    n = int(pl.shape[0])
    px = None if parent_x is None else _dev_u64(parent_x)
    m = min(int(K), 2 * n)
    if out is None:
        cx = torch.empty((max(m, 1), W), dtype=torch.int64, device=device)
        cl = torch.empty(max(m, 1), dtype=torch.float64, device=device)
        clt = torch.empty(max(m, 1), dtype=torch.float64, device=device)
    else:
        cx, cl, clt = out
        if cx.shape[0] < m or cx.shape[1] != W or cl.shape[0] < m or clt.shape[0] < m:
            raise ValueError("out has no room for min(K, 2 n_parents) vectors")
    nbytes = _GUMBEL_BYTES.get(n)
    if nbytes is None:
        nbytes = _GUMBEL_BYTES.setdefault(n, int(lib.nqs_gumbel_scratch_bytes(n)))
    if scratch is None:
        scratch = torch.empty(nbytes, dtype=torch.uint8, device=device)
    elif scratch.numel() < nbytes:
        raise ValueError("scratch is smaller than nqs_gumbel_scratch_bytes(n_parents)")
    else:
        nbytes = int(scratch.numel())
    out = ctypes.c_int64()
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(lib.nqs_gumbel_topk_level(int(n_qubits), int(level), n, None if px is None else px.data_ptr(),
                                     pl.data_ptr(), plt.data_ptr(), lp.data_ptr(), g.data_ptr(), int(K),
                                     scratch.data_ptr(), nbytes, cx.data_ptr(), cl.data_ptr(), clt.data_ptr(),
                                     ctypes.byref(out), s.cuda_stream))
    k = int(out.value)
    return cx[:k], cl[:k], clt[:k]


def gumbel_topk_level_async(n_qubits, level, max_parents, n_parents, parent_x, parent_l, parent_lt, cond_logp,
                            gumbel, K, out, scratch, counts, stream=None):
    """One qubit of Alg. 1 with the parent count on the device (nqs_gumbel_topk_level_async):
    no host synchronisation, so a run of levels can be enqueued or captured in a CUDA graph.

    n_parents: int64 CUDA tensor holding the count (the previous level's ``counts``, or 1);
    parent_l, parent_lt, cond_logp [.., 2], gumbel [.., 2]: FP64 CUDA tensors with at least
    max_parents rows; out = (child_x [.., W] int64, child_l, child_lt) with room for
    min(K, 2 max_parents); scratch: uint8 CUDA tensor of nqs_gumbel_scratch_bytes(max_parents);
    counts: int64 CUDA tensor [2] receiving (kept count, status 1 / 0 = a bucket overflowed)."""
    lib = _lib if _lib is not None else load_library()
    cx, cl, clt = out
    for t in (n_parents, parent_l, parent_lt, cond_logp, gumbel, cx, cl, clt, scratch, counts):
        if not (torch.is_tensor(t) and t.is_cuda and t.is_contiguous()):
            raise TypeError("the device-count form takes contiguous CUDA tensors only")
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(lib.nqs_gumbel_topk_level_async(int(n_qubits), int(level), int(max_parents), n_parents.data_ptr(),
                                           None if parent_x is None else parent_x.data_ptr(), parent_l.data_ptr(),
                                           parent_lt.data_ptr(), cond_logp.data_ptr(), gumbel.data_ptr(), int(K),
                                           scratch.data_ptr(), int(scratch.numel()), cx.data_ptr(), cl.data_ptr(),
                                           clt.data_ptr(), counts.data_ptr(), s.cuda_stream))


def ar_gumbel_topk(n_qubits, K, cond_logp, gumbel, device="cuda"):
    """Alg. 1 driven from the host: ``cond_logp(level, prefixes)`` -> [(log p(0|x), log p(1|x))]
    for the kept prefixes (Python ints), ``gumbel[level]`` -> the level's Gumbel draws (two per
    kept vector).  Returns (x [K', W] int64 tensor, l, L~) on the device, L~ descending."""
    W = (int(n_qubits) + 63) // 64
    x, l, lt = None, torch.zeros(1, dtype=torch.float64, device=device), torch.zeros(1, dtype=torch.float64,
                                                                                       device=device)
    for i in range(int(n_qubits)):
        if x is None:
            prefixes = [0]
        else:
            words = x.cpu().numpy().view(np.uint64)
            prefixes = [sum(int(words[r, w]) << (64 * w) for w in range(W)) for r in range(words.shape[0])]
        lp = np.asarray(cond_logp(i, prefixes), dtype=np.float64)
        g = np.asarray(gumbel[i], dtype=np.float64)[:2 * len(prefixes)]
        x, l, lt = gumbel_topk_level(n_qubits, i, x, l, lt, lp, g, K, device)
    return x, l, lt


def sr_top(logpsi_re, n_sr, stream=None):
    """Indices of the n_sr most probable samples (largest Re log psi; ties by index)."""
    lib = load_library()
    a = _f64(logpsi_re, "cuda")
    n = int(a.shape[0])
    nbytes = int(lib.nqs_sr_scratch_bytes(n, 1))
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=a.device)
    idx = torch.empty(min(int(n_sr), n), dtype=torch.int32, device=a.device)
    _check(lib.nqs_sr_top(n, _ptr(a), int(n_sr), _ptr(idx), _ptr(scratch), nbytes, _stream(stream)))
    return idx


def sr_step(O, logpsi_re, eloc_re, evar, lam, want_T=False, stream=None):
    """min-SR step on the GPU: (delta [n_params] FP64, T [n_sr, n_sr] FP64 or None).

    O: [n_sr, n_params] FP32 CUDA tensor of d log psi / d theta (real); evar: E
    (device tensor whose first entry is used, or a float)."""
    lib = load_library()
    O = O.to(dtype=torch.float32).contiguous()
    dev = O.device
    n, P = int(O.shape[0]), int(O.shape[1])
    a, el = _f64(logpsi_re, dev), _f64(eloc_re, dev)
    ev = _f64(evar if torch.is_tensor(evar) else np.array([float(evar)]), dev)
    nbytes = int(lib.nqs_sr_scratch_bytes(1, P))
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    delta = torch.empty(P, dtype=torch.float64, device=dev)
    T = torch.empty((n, n), dtype=torch.float64, device=dev) if want_T else None
    _check(lib.nqs_sr_step(n, P, _ptr(O), _ptr(a), _ptr(el), _ptr(ev), float(lam), _ptr(delta), _ptr(T), _ptr(scratch),
                           nbytes, _stream(stream)))
    return delta, T


class FullCandidates:
    """Candidates of the exact local energy (Eq. local_energy) for a staged batch.

    ``cand_id`` / ``hval``: [n_unq, n_xy] (int32 holding uint32 candidate
    indices, FP64 matrix elements), ``cand``: [n_cand, W] distinct candidates
    in increasing numeric order, ``in_u``: index of each candidate in U or -1.
    """

    def __init__(self, batch, cand_id, hval, cand, in_u, scratch):
        self.batch, self.cand_id, self.hval, self.cand, self.in_u = batch, cand_id, hval, cand, in_u
        self.scratch = scratch

    @property
    def n_cand(self):
        return int(self.cand.shape[0])


def full_candidates(batch: Batch, with_h=True, stream=None):
    """Every x XOR XY of every sample, deduplicated over the batch (nqs_full_candidates)."""
    lib = load_library()
    ham = batch.ham
    n_xy = int(ham.info["n_xy"])
    dev = batch.device
    nbytes = int(lib.nqs_candidates_scratch_bytes(ham.handle, batch.n))
    if nbytes < 0:
        _check(nbytes)
    scratch = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=dev)
    cand_id = torch.empty((batch.n, n_xy), dtype=torch.int32, device=dev)
    hval = torch.empty((batch.n, n_xy), dtype=torch.float64, device=dev) if with_h else None
    n = ctypes.c_int64()
    # the candidate count of the last call on this batch (a retry reruns the whole pipeline)
    cap = getattr(batch, "_cand_cap", None) or max(batch.n * n_xy // 4, 1024)
    for _ in range(2):
        cand = torch.empty((cap, ham.n_words), dtype=torch.int64, device=dev)
        in_u = torch.empty(cap, dtype=torch.int32, device=dev)
        rc = lib.nqs_full_candidates(ham.handle, _ptr(batch.U), batch.n, _ptr(batch.work), _ptr(scratch),
                                     scratch.numel(), _ptr(cand_id), _ptr(hval), _ptr(cand), _ptr(in_u), cap,
                                     ctypes.byref(n), _stream(stream))
        if rc == -4 and n.value > cap:
            cap = int(n.value)
            batch._cand_cap = cap
            continue
        _check(rc)
        break
    k = int(n.value)
    return FullCandidates(batch, cand_id, hval, cand[:k], in_u[:k], scratch)


def local_energy_full(fc: FullCandidates, logpsi_re, logpsi_im, cand_logpsi_re, cand_logpsi_im=None,
                      out=None, stream=None):
    """Exact E_loc (Eq. local_energy) from the candidates' log-amplitudes: (eloc_re, eloc_im or None)."""
    batch = fc.batch
    dev = batch.device
    a, b = _f64(logpsi_re, dev), _f64(logpsi_im, dev)
    ca, cb = _f64(cand_logpsi_re, dev), _f64(cand_logpsi_im, dev)
    cplx = b is not None or cb is not None
    if out is None:
        er = torch.empty(batch.n, dtype=torch.float64, device=dev)
        ei = torch.empty(batch.n, dtype=torch.float64, device=dev) if cplx else None
    else:
        er, ei = out
    _check(_lib.nqs_local_energy_full(batch.ham.handle, _ptr(batch.U), batch.n, _ptr(batch.work), _ptr(a), _ptr(b),
                                      _ptr(fc.cand_id), _ptr(fc.hval), fc.n_cand, _ptr(ca), _ptr(cb),
                                      _ptr(fc.scratch), fc.scratch.numel(), _ptr(er), _ptr(ei), _stream(stream)))
    return er, ei


class _Instance(ctypes.Structure):
    _fields_ = [("ham", ctypes.c_void_p), ("U", ctypes.c_void_p), ("n_unq", ctypes.c_int64),
                ("logpsi_re", ctypes.c_void_p), ("eloc_re", ctypes.c_void_p), ("evar", ctypes.c_void_p),
                ("grad", ctypes.c_void_p)]


class BatchedPlan:
    """Many independent (Hamiltonian, batch) instances evaluated by one CUDA-graph launch.

    ``items``: list of (Hamiltonian, U, logpsi_re).  ``U`` and ``logpsi_re``
    are kept as device tensors whose contents may be overwritten between
    runs (same sizes).  ``run()`` launches the graph asynchronously; results
    are ``eloc[i]`` (E_loc^var) and ``evar[i]`` ([E^var, max log psi, sum of
    weights]).  ``autotune`` times the pair-search schedules and their launch
    parameters per instance at planning time.  With ``gradients`` every run
    also writes ``grad[i]`` = dE^var / d Re log psi (the adjoint's closed form).
    """

    def __init__(self, items, precision="fp32c", autotune=True, gradients=False, stream=None):
        lib = load_library()
        self.hams, self.U, self.logpsi, self.eloc, self.evar, self.grad = [], [], [], [], [], []
        arr = (_Instance * len(items))()
        for i, (ham, U, lre) in enumerate(items):
            Ud = _dev_u64(U)
            if Ud.shape[1] != ham.n_words:
                raise ValueError(f"instance {i}: word count does not match its Hamiltonian")
            a = _f64(lre, Ud.device)
            er = torch.zeros(Ud.shape[0], dtype=torch.float64, device=Ud.device)
            ev = torch.zeros(3, dtype=torch.float64, device=Ud.device)
            gr = torch.zeros(Ud.shape[0], dtype=torch.float64, device=Ud.device) if gradients else None
            self.hams.append(ham); self.U.append(Ud); self.logpsi.append(a)
            self.eloc.append(er); self.evar.append(ev); self.grad.append(gr)
            arr[i] = _Instance(ham.handle.value, Ud.data_ptr(), Ud.shape[0], a.data_ptr(), er.data_ptr(),
                               ev.data_ptr(), None if gr is None else gr.data_ptr())
        h = ctypes.c_void_p()
        _check(lib.nqs_batch_plan(arr, len(items), PRECISIONS[precision], 1 if autotune else 0,
                                  ctypes.byref(h), _stream(stream)))
        self._h = h

    def run(self, stream=None):
        _check(_lib.nqs_batch_run(self._h, _stream(stream)))

    def status(self, stream=None):
        bad = ctypes.c_int()
        rc = _lib.nqs_batch_status(self._h, ctypes.byref(bad), _stream(stream))
        return rc, int(bad.value)

    def info(self, i):
        v = (ctypes.c_int64 * 8)()
        _check(_lib.nqs_batch_info(self._h, int(i), v))
        sched = {v2: k for k, v2 in SCHEDULES.items()}[int(v[0])]
        t = (ctypes.c_int32 * 3)()
        _check(_lib.nqs_batch_tune(self._h, int(i), t))
        return {"schedule": sched, "capacity": v[1], "planned_pairs": v[2], "graph_nodes": v[3],
                "t_terms_us": v[4], "t_batch_us": v[5], "t_trie_us": v[6], "graph_kernels": v[7],
                "tune": {"terms_grab": t[0], "terms_groups": t[1], "trie_pop": t[2]}}

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.nqs_batch_free(self._h)
            self._h = None
