"""Thin ctypes binding of libdf (include/df.h): argument marshalling only.

Every step of the J/K builds runs in the CUDA library; this module only turns
torch CUDA tensors into device pointers and the current stream into a
``cudaStream_t``.  There is no CPU fallback: if ``_build/libdf.so`` is missing
or CUDA is unavailable, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdf.so")

S_MAX = 8
AUX_BLOCK = 128
OPT_CLUSTER_PAIRS = 1  # DF_OPT_CLUSTER_PAIRS
OPT_SPARSE = 2         # DF_OPT_SPARSE
OPT_JK_OVERLAP = 3     # DF_OPT_JK_OVERLAP
PHASES = ("split_C", "gemm1", "split_X", "gemm2", "reduce", "rho", "coulomb", "energy")

_STATUS = {0: "ok", -1: "invalid argument", -2: "CUDA or cuBLAS call failed", -3: "device allocation failed",
           -4: "metric not positive definite", -5: "bounded device wait ran out", -6: "result missed its tolerance",
           -7: "call out of order", -8: "problem exceeds the static scratch of df_emulated_gemm_static"}


class DFError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__("%s: %s (status %d)" % (where, _STATUS.get(status, "unknown"), status))
        self.status = status


ADAPTIVE = -1  # df_build_K: the count of the context's current Table 1 level
LEARNED = -2   # df_build_K: per-block counts from the attached network, checked


class KStats(ctypes.Structure):
    _fields_ = [("nblk", ctypes.c_int), ("slices", ctypes.c_int * 256), ("recomputed", ctypes.c_int),
                ("fallback", ctypes.c_int), ("low_confidence", ctypes.c_int), ("level", ctypes.c_int),
                ("slice_pairs", ctypes.c_longlong), ("bound_ratio", ctypes.c_double)]

    def as_dict(self):
        n = min(self.nblk, 256)
        return {"nblk": self.nblk, "slices": list(self.slices[:n]), "recomputed": self.recomputed,
                "fallback": self.fallback, "low_confidence": self.low_confidence, "level": self.level,
                "slice_pairs": self.slice_pairs, "bound_ratio": self.bound_ratio}


_lib = None


def lib():
    """Load libdf; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libdf is not built (%s missing): run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        pp = ctypes.POINTER(ctypes.c_void_p)
        L.df_create.argtypes = [pp, I, I, I, I]
        L.df_destroy.argtypes = [P]
        L.df_destroy.restype = None
        L.df_setup.argtypes = [P, P, V]
        L.df_setup_ordered.argtypes = [P, P, ctypes.POINTER(ctypes.c_int), V]
        L.df_setup_integrals.argtypes = [P, P, P, ctypes.POINTER(ctypes.c_int), V]
        L.df_setup_packed.argtypes = [P, P, ctypes.POINTER(ctypes.c_int), V]
        L.df_build_J.argtypes = [P, P, P, P, V]
        L.df_build_K.argtypes = [P, P, I, I, P, ctypes.POINTER(KStats), V]
        L.df_build_JK.argtypes = [P, P, P, I, I, P, P, P, ctypes.POINTER(KStats), V]
        L.df_build_K_blocks.argtypes = [P, P, I, ctypes.POINTER(ctypes.c_int), P, ctypes.POINTER(KStats), V]
        L.df_energy.argtypes = [P, P, P, P, P, ctypes.POINTER(ctypes.c_double), V]
        L.df_split_int8.argtypes = [P, I, I, I, I, P, P, V]
        L.df_slice_products.argtypes = [P, P, I, I, I, I, P, P, P, V]
        L.df_emulated_gemm.argtypes = [P, P, I, I, I, I, P, V]
        L.df_level_for.argtypes = [D]
        L.df_level_for.restype = I
        L.df_level_slices.argtypes = [I]
        L.df_level_slices.restype = I
        L.df_adaptive_reset.argtypes = [P, I]
        L.df_adaptive_level0.argtypes = [P, I]
        L.df_adaptive_next.argtypes = [P, D, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.df_sync_status.argtypes = [P, V]
        L.df_selftest_wait_timeout.argtypes = [I, V]
        L.df_last_error.argtypes = [P]
        L.df_strerror.argtypes = [I]
        L.df_strerror.restype = ctypes.c_char_p
        L.df_set_profiling.argtypes = [P, I]
        L.df_set_option.argtypes = [P, I, I]
        L.df_phase_times.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
        PP = ctypes.POINTER(ctypes.c_void_p)
        L.df_batch_create.argtypes = [pp, PP, I]
        L.df_batch_destroy.argtypes = [P]
        L.df_batch_destroy.restype = None
        L.df_batch_set_graphs.argtypes = [P, I]
        L.df_batch_build_K.argtypes = [P, PP, ctypes.POINTER(ctypes.c_int), I, PP, V]
        L.df_batch_build_J.argtypes = [P, PP, PP, V]
        L.df_batch_autotune.argtypes = [P, PP, ctypes.POINTER(ctypes.c_int), I, PP, V, ctypes.POINTER(ctypes.c_int)]
        FP = ctypes.POINTER(ctypes.c_float)
        L.df_mlp_create.argtypes = [pp]
        L.df_mlp_destroy.argtypes = [P]
        L.df_mlp_destroy.restype = None
        L.df_mlp_num_params.argtypes = []
        L.df_mlp_set_params.argtypes = [P, FP, I]
        L.df_mlp_get_params.argtypes = [P, FP, I]
        L.df_mlp_forward.argtypes = [P, P, I, P, V]
        L.df_mlp_gradients.argtypes = [P, P, P, I, FP, FP, V]
        L.df_mlp_train_step.argtypes = [P, P, P, I, ctypes.c_float, FP, V]
        L.df_block_features.argtypes = [P, I, D, D, D, I, P, V]
        L.df_block_errors.argtypes = [P, P, I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), V]
        L.df_set_predictor.argtypes = [P, P, ctypes.c_float]
        L.df_sparsity.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        L.df_workspace_bytes.argtypes = [P]
        L.df_workspace_bytes.restype = ctypes.c_int64
        LL = ctypes.c_longlong
        L.df_crt_modulus.argtypes = [I]
        L.df_crt_operand_bits.argtypes = [LL, I]
        L.df_crt_moduli_for_bits.argtypes = [LL, I]
        L.df_crt_split_rows.argtypes = [P, I, I, I, I, P, P, V]
        L.df_crt_residue_products.argtypes = [P, P, I, I, I, I, P, P, P, V]
        L.df_emulated_gemm_crt.argtypes = [P, P, I, I, I, I, P, V]
        _lib = L
    return _lib


def _check(status: int, where: str) -> None:
    if status != 0:
        raise DFError(status, where)


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _f64(t):
    if t.dtype != torch.float64:
        raise ValueError("expected float64, got %s" % t.dtype)
    return _ptr(t)


def level_for(dE_rel: float) -> int:
    return lib().df_level_for(float(dE_rel))


def level_slices(level: int) -> int:
    return lib().df_level_slices(int(level))


def split_int8(A: torch.Tensor, nslices: int, stream=None):
    """Row exponents (int32) and INT8 digits [nslices, rows, cols] of a 2-D FP64 tensor."""
    rows, cols = A.shape
    exps = torch.empty(rows, dtype=torch.int32, device=A.device)
    digits = torch.empty((nslices, rows, cols), dtype=torch.int8, device=A.device)
    _check(lib().df_split_int8(_f64(A), rows, cols, cols, nslices, _ptr(exps), _ptr(digits), _stream(stream)),
           "df_split_int8")
    return exps, digits


def slice_products(A: torch.Tensor, B: torch.Tensor, nslices: int, stream=None):
    """Exact S_g = sum_{t+u=g} A_t B_u^T, returned as int64 [nslices, M, N], plus row exponents."""
    M, K = A.shape
    N, K2 = B.shape
    assert K == K2
    S = torch.empty((nslices, N, M), dtype=torch.int64, device=A.device)
    ea = torch.empty(M, dtype=torch.int32, device=A.device)
    eb = torch.empty(N, dtype=torch.int32, device=A.device)
    _check(lib().df_slice_products(_f64(A), _f64(B), M, N, K, nslices, _ptr(S), _ptr(ea), _ptr(eb),
                                   _stream(stream)), "df_slice_products")
    return S.transpose(1, 2), ea, eb


def emulated_gemm(A: torch.Tensor, B: torch.Tensor, nslices: int, stream=None):
    """A @ B^T emulated with nslices INT8 slices per operand."""
    M, K = A.shape
    N, _ = B.shape
    out = torch.empty((M, N), dtype=torch.float64, device=A.device)
    _check(lib().df_emulated_gemm(_f64(A), _f64(B), M, N, K, nslices, _ptr(out), _stream(stream)),
           "df_emulated_gemm")
    return out


def selftest_wait_timeout(limit_ms: int = 1000, stream=None) -> int:
    """Run the bounded-wait failure self-test; returns its status (DF_ERR_TIMEOUT = -5 expected)."""
    return lib().df_selftest_wait_timeout(int(limit_ms), _stream(stream))


def crt_modulus(i: int) -> int:
    return lib().df_crt_modulus(int(i))


def crt_operand_bits(K: int, nmod: int) -> int:
    return lib().df_crt_operand_bits(int(K), int(nmod))


def crt_moduli_for_bits(K: int, bits: int) -> int:
    return lib().df_crt_moduli_for_bits(int(K), int(bits))


def crt_split_rows(A: torch.Tensor, nmod: int, stream=None):
    """Row exponents (int32) and centred residues int16 [nmod, rows, cols] of the scaled rows of A."""
    rows, cols = A.shape
    exps = torch.empty(rows, dtype=torch.int32, device=A.device)
    res = torch.empty((nmod, rows, cols), dtype=torch.int16, device=A.device)
    _check(lib().df_crt_split_rows(_f64(A), rows, cols, cols, nmod, _ptr(exps), _ptr(res), _stream(stream)),
           "df_crt_split_rows")
    return exps, res


def crt_residue_products(A: torch.Tensor, B: torch.Tensor, nmod: int, stream=None):
    """y_i = (a_i b_i^T) mod m_i as uint8 [nmod, M, N], plus the row exponents of A and B."""
    M, K = A.shape
    N, _ = B.shape
    Y = torch.empty((nmod, M, N), dtype=torch.uint8, device=A.device)
    ea = torch.empty(M, dtype=torch.int32, device=A.device)
    eb = torch.empty(N, dtype=torch.int32, device=A.device)
    _check(lib().df_crt_residue_products(_f64(A), _f64(B), M, N, K, nmod, _ptr(Y), _ptr(ea), _ptr(eb),
                                         _stream(stream)), "df_crt_residue_products")
    return Y, ea, eb


def emulated_gemm_crt(A: torch.Tensor, B: torch.Tensor, nmod: int, stream=None):
    """A @ B^T emulated through the residues of nmod moduli (CRT variant)."""
    M, K = A.shape
    N, _ = B.shape
    out = torch.empty((M, N), dtype=torch.float64, device=A.device)
    _check(lib().df_emulated_gemm_crt(_f64(A), _f64(B), M, N, K, nmod, _ptr(out), _stream(stream)),
           "df_emulated_gemm_crt")
    return out


class Context:
    """One molecule's DF workspaces on the current CUDA device."""

    def __init__(self, nao: int, naux: int, nocc_max: int, s_max: int = S_MAX):
        self.nao, self.naux, self.nocc_max, self.s_max = nao, naux, nocc_max, s_max
        self.nblk = (naux + AUX_BLOCK - 1) // AUX_BLOCK
        h = ctypes.c_void_p()
        _check(lib().df_create(ctypes.byref(h), nao, naux, nocc_max, s_max), "df_create")
        self._h = h
        self._B = None

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().df_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def workspace_bytes(self) -> int:
        return int(lib().df_workspace_bytes(self._h))

    def sparsity(self):
        """(nonzero K-tile fraction of the first GEMM, nonzero (mu, 64-nu chunk) fraction of rho/J)."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(lib().df_sparsity(self._h, ctypes.byref(a), ctypes.byref(b)), "df_sparsity")
        return a.value, b.value

    def setup(self, B: torch.Tensor, perm=None, stream=None):
        """Attach B; `perm` (new position -> original P) orders the exchange path's auxiliary functions."""
        assert B.shape == (self.naux, self.nao, self.nao)
        self._B = B  # the library keeps the pointer: keep the tensor alive
        if perm is None:
            _check(lib().df_setup(self._h, _f64(B), _stream(stream)), "df_setup")
        else:
            arr = (ctypes.c_int * self.naux)(*[int(x) for x in perm])
            _check(lib().df_setup_ordered(self._h, _f64(B), arr, _stream(stream)), "df_setup_ordered")

    def setup_packed(self, Bp: torch.Tensor, perm=None, stream=None):
        """Attach B given as packed upper triangles [naux, nao (nao + 1) / 2] (see inputs.pack_upper)."""
        assert Bp.shape == (self.naux, self.nao * (self.nao + 1) // 2)
        self._B = Bp
        arr = None if perm is None else (ctypes.c_int * self.naux)(*[int(x) for x in perm])
        _check(lib().df_setup_packed(self._h, _f64(Bp), arr, _stream(stream)), "df_setup_packed")

    def setup_integrals(self, T: torch.Tensor, V: torch.Tensor, perm=None, stream=None):
        """Form B = L^{-1} T in place on the device (L L^T = V) and attach it; returns T (now B)."""
        assert T.shape == (self.naux, self.nao, self.nao) and V.shape == (self.naux, self.naux)
        assert T.dtype == torch.float64 and V.dtype == torch.float64 and T.is_contiguous() and V.is_contiguous()
        self._B = T
        arr = None if perm is None else (ctypes.c_int * self.naux)(*[int(x) for x in perm])
        _check(lib().df_setup_integrals(self._h, _f64(T), _f64(V), arr, _stream(stream)), "df_setup_integrals")
        return T

    def build_J(self, D, J=None, rho=None, stream=None):
        if J is None:
            J = torch.empty((self.nao, self.nao), dtype=torch.float64, device=D.device)
        if rho is None:
            rho = torch.empty(self.naux, dtype=torch.float64, device=D.device)
        _check(lib().df_build_J(self._h, _f64(D), _f64(J), _f64(rho), _stream(stream)), "df_build_J")
        return J, rho

    def set_predictor(self, mlp, min_conf: float = 0.6):
        """Attach a network for build_K(C, LEARNED) (None detaches); the context keeps the pointer."""
        self._pred = mlp
        _check(lib().df_set_predictor(self._h, None if mlp is None else mlp._h, float(min_conf)), "df_set_predictor")

    def build_K(self, C, nslices: int, K=None, stream=None):
        """nslices: 1..8 fixed, 0 native FP64, ADAPTIVE (-1) the current level's count, LEARNED (-2)."""
        nocc = C.shape[1]
        if K is None:
            K = torch.empty((self.nao, self.nao), dtype=torch.float64, device=C.device)
        st = KStats()
        _check(lib().df_build_K(self._h, _f64(C), nocc, int(nslices), _f64(K), ctypes.byref(st), _stream(stream)),
               "df_build_K")
        return K, st

    def build_JK(self, D, C, nslices: int, J=None, rho=None, K=None, stream=None):
        """build_J(D) then build_K(C, nslices) in one call (rho and J beside the X split); (J, rho, K, stats)."""
        nocc = C.shape[1]
        if J is None:
            J = torch.empty((self.nao, self.nao), dtype=torch.float64, device=D.device)
        if rho is None:
            rho = torch.empty(self.naux, dtype=torch.float64, device=D.device)
        if K is None:
            K = torch.empty((self.nao, self.nao), dtype=torch.float64, device=C.device)
        st = KStats()
        _check(lib().df_build_JK(self._h, _f64(D), _f64(C), nocc, int(nslices), _f64(J), _f64(rho), _f64(K),
                                 ctypes.byref(st), _stream(stream)), "df_build_JK")
        return J, rho, K, st

    def build_K_blocks(self, C, slices, K=None, stream=None):
        nocc = C.shape[1]
        if K is None:
            K = torch.empty((self.nao, self.nao), dtype=torch.float64, device=C.device)
        arr = (ctypes.c_int * self.nblk)(*[int(s) for s in slices])
        st = KStats()
        _check(lib().df_build_K_blocks(self._h, _f64(C), nocc, arr, _f64(K), ctypes.byref(st), _stream(stream)),
               "df_build_K_blocks")
        return K, st

    def energy(self, D, J=None, K=None, rho=None, stream=None):
        """(1/2 tr DJ, 1/2 rho.rho, -1/2 tr DK); synchronises the stream."""
        E = (ctypes.c_double * 3)()
        _check(lib().df_energy(self._h, _f64(D), _ptr(J), _ptr(K), _ptr(rho), E, _stream(stream)), "df_energy")
        return E[0], E[1], E[2]

    def adaptive_reset(self, fp64_from_level: int = -1):
        _check(lib().df_adaptive_reset(self._h, int(fp64_from_level)), "df_adaptive_reset")

    def adaptive_level0(self, nslices: int):
        _check(lib().df_adaptive_level0(self._h, int(nslices)), "df_adaptive_level0")

    def adaptive_next(self, energy: float):
        lv, ns = ctypes.c_int(), ctypes.c_int()
        _check(lib().df_adaptive_next(self._h, float(energy), ctypes.byref(lv), ctypes.byref(ns)),
               "df_adaptive_next")
        return lv.value, ns.value

    def set_profiling(self, on: bool):
        _check(lib().df_set_profiling(self._h, 1 if on else 0), "df_set_profiling")

    def set_cluster_pairs(self, mode: int):
        """DF_OPT_CLUSTER_PAIRS: 0 never, 1 the first exchange GEMM (default), 2 both GEMMs."""
        _check(lib().df_set_option(self._h, OPT_CLUSTER_PAIRS, int(mode)), "df_set_option")

    def set_sparse(self, on: bool):
        """DF_OPT_SPARSE: use the block sparsity of a screened B (default) or run dense."""
        _check(lib().df_set_option(self._h, OPT_SPARSE, 1 if on else 0), "df_set_option")

    def set_jk_overlap(self, ctas_per_sm: int):
        """DF_OPT_JK_OVERLAP: CTAs per SM of rho and J beside the X split in build_JK (0 = in order)."""
        _check(lib().df_set_option(self._h, OPT_JK_OVERLAP, int(ctas_per_sm)), "df_set_option")

    def phase_times(self):
        """{phase: (total ms, records)} since the last read (waits for the events)."""
        ms = (ctypes.c_double * len(PHASES))()
        cnt = (ctypes.c_int * len(PHASES))()
        _check(lib().df_phase_times(self._h, ms, cnt), "df_phase_times")
        return {name: (ms[i], cnt[i]) for i, name in enumerate(PHASES)}

    def sync_status(self, stream=None):
        _check(lib().df_sync_status(self._h, _stream(stream)), "df_sync_status")


def _ptr_array(tensors):
    arr = (ctypes.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        arr[i] = _f64(t)
    return arr


class Batch:
    """Batched J/K builds over several contexts (grouped persistent launches + CUDA graphs)."""

    def __init__(self, contexts):
        self.contexts = list(contexts)
        handles = (ctypes.c_void_p * len(self.contexts))(*[c._h.value for c in self.contexts])
        h = ctypes.c_void_p()
        _check(lib().df_batch_create(ctypes.byref(h), handles, len(self.contexts)), "df_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().df_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_graphs(self, on: bool):
        _check(lib().df_batch_set_graphs(self._h, 1 if on else 0), "df_batch_set_graphs")

    def build_K(self, Cs, nslices: int, Ks, stream=None):
        nocc = (ctypes.c_int * len(Cs))(*[int(C.shape[1]) for C in Cs])
        _check(lib().df_batch_build_K(self._h, _ptr_array(Cs), nocc, int(nslices), _ptr_array(Ks), _stream(stream)),
               "df_batch_build_K")

    def build_J(self, Ds, Js, stream=None):
        _check(lib().df_batch_build_J(self._h, _ptr_array(Ds), _ptr_array(Js), _stream(stream)), "df_batch_build_J")

    def autotune(self, Cs, nslices: int, Ks, stream=None):
        nocc = (ctypes.c_int * len(Cs))(*[int(C.shape[1]) for C in Cs])
        ch = (ctypes.c_int * 3)()
        _check(lib().df_batch_autotune(self._h, _ptr_array(Cs), nocc, int(nslices), _ptr_array(Ks), _stream(stream),
                                       ch), "df_batch_autotune")
        return ch[0], ch[1], ch[2]


class MLP:
    """The slice-count predictor network on the device (16 -> 64 -> 64 -> 8)."""

    def __init__(self, params=None):
        h = ctypes.c_void_p()
        _check(lib().df_mlp_create(ctypes.byref(h)), "df_mlp_create")
        self._h = h
        self.n_params = lib().df_mlp_num_params()
        if params is not None:
            self.set_params(params)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().df_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        import numpy as np
        a = np.ascontiguousarray(params, dtype=np.float32)
        assert a.size == self.n_params
        _check(lib().df_mlp_set_params(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size),
               "df_mlp_set_params")

    def get_params(self):
        import numpy as np
        a = np.empty(self.n_params, dtype=np.float32)
        _check(lib().df_mlp_get_params(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size),
               "df_mlp_get_params")
        return a

    def forward(self, X, stream=None):
        assert X.dtype == torch.float32 and X.shape[1] == 16
        probs = torch.empty((X.shape[0], 8), dtype=torch.float32, device=X.device)
        _check(lib().df_mlp_forward(self._h, _ptr(X), X.shape[0], _ptr(probs), _stream(stream)), "df_mlp_forward")
        return probs

    def gradients(self, X, y, stream=None):
        import numpy as np
        g = np.empty(self.n_params, dtype=np.float32)
        loss = ctypes.c_float()
        _check(lib().df_mlp_gradients(self._h, _ptr(X), _ptr(y), X.shape[0],
                                      g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(loss),
                                      _stream(stream)), "df_mlp_gradients")
        return g, loss.value

    def train_step(self, X, y, lr, want_loss=False, stream=None):
        loss = ctypes.c_float()
        _check(lib().df_mlp_train_step(self._h, _ptr(X), _ptr(y), X.shape[0], float(lr),
                                       ctypes.byref(loss) if want_loss else None, _stream(stream)),
               "df_mlp_train_step")
        return loss.value if want_loss else None


def block_features(ctx, nocc, tau, dD, dE, s_rule, stream=None):
    F = torch.empty((ctx.nblk, 16), dtype=torch.float32, device="cuda")
    _check(lib().df_block_features(ctx._h, int(nocc), float(tau), float(dD), float(dE), int(s_rule), _ptr(F),
                                   _stream(stream)), "df_block_features")
    return F


def block_errors(ctx, C, stream=None):
    """(err [nblk, 8] max|K_b(s) - K_b(FP64)| for s = 1..8, max|K(FP64)|)."""
    import numpy as np
    err = np.zeros((ctx.nblk, 8))
    kmax = ctypes.c_double()
    _check(lib().df_block_errors(ctx._h, _f64(C), C.shape[1], err.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 ctypes.byref(kmax), _stream(stream)), "df_block_errors")
    return err, kmax.value
