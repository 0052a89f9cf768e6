"""ctypes binding of the bps C ABI (include/bps.h): argument marshalling only.

Every function here has the name of the C entry point it wraps.  Field
arguments are torch CUDA tensors (their device pointers are passed through);
scalar arrays are numpy / Python sequences.  A missing or unloadable library
raises: there is no fallback path.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libbps.so")

BPS_OK, BPS_EINVAL, BPS_ENOMEM, BPS_ECUDA, BPS_ENUMERIC, BPS_ETIMEOUT, BPS_ESTATE = range(7)
STATUS_NAMES = ["BPS_OK", "BPS_EINVAL", "BPS_ENOMEM", "BPS_ECUDA", "BPS_ENUMERIC", "BPS_ETIMEOUT", "BPS_ESTATE"]


class BpsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class bps_config(ctypes.Structure):
    _fields_ = [("n_bins", ctypes.c_int), ("alpha", ctypes.c_double), ("n_leapfrog", ctypes.c_int),
                ("eps_max", ctypes.c_double), ("jump", ctypes.c_int), ("jump_leapfrog", ctypes.c_int),
                ("jump_eps_max", ctypes.c_double), ("fixed_bias_index", ctypes.c_int),
                ("mass_mode", ctypes.c_int), ("seed", ctypes.c_uint64)]


class bps_schechter(ctypes.Structure):
    _fields_ = [("M_star", ctypes.c_double), ("alpha", ctypes.c_double), ("m_bright", ctypes.c_double),
                ("m_faint", ctypes.c_double), ("omega_m", ctypes.c_double)]


# the paper's Schechter and survey parameters (Sec. 5)
SCHECHTER_SDSS = dict(M_star=-20.44, alpha=-1.05, m_bright=14.5, m_faint=17.77, omega_m=0.24)
BIAS_LAW_PAPER = dict(b_star=1.2, M_star=-20.83, a=0.895, b=0.105, c=-0.040)


class bps_move_info(ctypes.Structure):
    _fields_ = [("accepted", ctypes.c_int), ("dH", ctypes.c_double), ("eps", ctypes.c_double)]


_lib = None

_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "bps_create": ([ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.POINTER(bps_config), _P,
                    ctypes.POINTER(_P)], ctypes.c_int),
    "bps_set_data": ([_P, _P, _P], ctypes.c_int),
    "bps_set_data_host": ([_P, _P, _P], ctypes.c_int),
    "bps_set_data_host_u16": ([_P, _P, _P], ctypes.c_int),
    "bps_stage_data_host_u16": ([_P, _P, _P], ctypes.c_int),
    "bps_z_line_pairs": ([_P], ctypes.c_int),
    "bps_x_pass_variant": ([_P], ctypes.c_int),
    "bps_adapt_step_size": ([_P, ctypes.c_int, ctypes.c_int, ctypes.c_double, _D], ctypes.c_int),
    "bps_set_preconditioner": ([_P, _P, ctypes.c_size_t], ctypes.c_int),
    "bps_mlp_export": ([_P, _P, _P, ctypes.c_double, _P, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "bps_set_state": ([_P, _P, _D, _D, _D, ctypes.c_uint64], ctypes.c_int),
    "bps_get_state": ([_P, _P, _D, _D, _D, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "bps_get_spectrum": ([_P, _P], ctypes.c_int),
    "bps_set_spectrum": ([_P, _P], ctypes.c_int),
    "bps_hmc_step": ([_P, ctypes.POINTER(bps_move_info)], ctypes.c_int),
    "bps_sample_power": ([_P, _D, _D], ctypes.c_int),
    "bps_sample_bias_norm": ([_P, _D, _D, _D], ctypes.c_int),
    "bps_jump": ([_P, ctypes.POINTER(bps_move_info)], ctypes.c_int),
    "bps_gibbs_iterate": ([_P, ctypes.c_int, _D], ctypes.c_int),
    "bps_set_mass_scale": ([_P, ctypes.c_int, _D], ctypes.c_int),
    "bps_fft_r2c": ([_P, _P, _P], ctypes.c_int),
    "bps_fft_c2r": ([_P, _P, _P], ctypes.c_int),
    "bps_gradient": ([_P, _P, _D], ctypes.c_int),
    "bps_philox_words": ([ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                          ctypes.c_size_t, _P, _P], ctypes.c_int),
    "bps_voxel_normals": ([ctypes.c_uint64, ctypes.c_uint64, ctypes.c_size_t, _P, _P], ctypes.c_int),
    "bps_version": ([], ctypes.c_char_p),
    "bps_last_error": ([_P], ctypes.c_char_p),
    "bps_kernel_launches": ([_P], ctypes.c_uint64),
    "bps_profile": ([_P, ctypes.c_int], ctypes.c_int),
    "bps_profile_read": ([_P, _D, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "bps_create_batch": ([ctypes.c_int, _P, _P, _P, ctypes.POINTER(bps_config), _P, ctypes.POINTER(_P)], ctypes.c_int),
    "bps_batch_set_chain": ([_P, ctypes.c_int, _P, _P, _P, _D, _D, _D, ctypes.c_uint64], ctypes.c_int),
    "bps_batch_get_chain": ([_P, ctypes.c_int, _P, _D, _D, _D, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "bps_batch_gibbs_iterate": ([_P, ctypes.c_int, _D], ctypes.c_int),
    "bps_batch_record_len": ([_P], ctypes.c_int),
    "bps_batch_record_slot": ([_P, ctypes.c_int], ctypes.c_int),
    "bps_mlp_create": ([ctypes.c_int, _P, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "bps_mlp_num_params": ([_P], ctypes.c_size_t),
    "bps_mlp_set_params": ([_P, _P], ctypes.c_int),
    "bps_mlp_get_params": ([_P, _P], ctypes.c_int),
    "bps_mlp_forward": ([_P, ctypes.c_int, _P, _P], ctypes.c_int),
    "bps_mlp_loss_grad": ([_P, ctypes.c_int, _P, _P, _D, _P], ctypes.c_int),
    "bps_mlp_adam_step": ([_P, ctypes.c_float], ctypes.c_int),
    "bps_mlp_train": ([_P, ctypes.c_int, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_uint64, _D],
                      ctypes.c_int),
    "bps_mlp_destroy": ([_P], None),
    "bps_mass_stats": ([_P, ctypes.c_int, ctypes.c_int, _D], ctypes.c_int),
    "bps_window_power": ([_P, _D], ctypes.c_int),
    "bps_set_mass_net": ([_P, _P, _P, _P, ctypes.c_double], ctypes.c_int),
    "bps_get_mass_scale": ([_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _D], ctypes.c_int),
    "bps_bin_power_noalloc": ([ctypes.c_int, ctypes.c_double, ctypes.c_int, _P, _P, _P], ctypes.c_int),
    "bps_save_chain": ([_P, _P, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "bps_load_chain": ([_P, _P, ctypes.c_size_t], ctypes.c_int),
    "bps_selftest_wait": ([_P, ctypes.c_uint64], ctypes.c_int),
    "bps_posterior_moments": ([_P, ctypes.c_int], ctypes.c_int),
    "bps_posterior_read": ([_P, _P, _P, _D, _D, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "bps_mock_field": ([_P, ctypes.c_uint64, _D, _P], ctypes.c_int),
    "bps_mock_counts": ([_P, ctypes.c_uint64, _P, _P, _D, _D, ctypes.c_int, _P], ctypes.c_int),
    "bps_mock_response": ([_P, ctypes.c_double, _D, ctypes.c_int, _D, _P], ctypes.c_int),
    "bps_schechter_tables": ([ctypes.POINTER(bps_schechter), ctypes.c_int, _D, ctypes.c_double, ctypes.c_int, _D,
                              _D], ctypes.c_int),
    "bps_bias_law": ([ctypes.c_int, _D, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                      ctypes.c_double, _D], ctypes.c_int),
    "bps_destroy": ([_P], None),
}


def load(path=None):
    """Load libbps.so (built by paper_1306_1821_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise FileNotFoundError(f"{p} not found: build it with paper_1306_1821_gb300.build.build()")
    lib = ctypes.CDLL(p)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def declared_symbols():
    return list(_SIGS)


def _dptr(t):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _darr(x, n=None):
    if x is None:
        return None, None
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None and a.size < n:
        raise ValueError("array too short")
    return a, a.ctypes.data_as(_D)


def _check(ctx, status):
    if status != BPS_OK:
        msg = load().bps_last_error(ctx)
        raise BpsError(status, msg.decode() if msg else "")


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def make_config(n_bins, alpha=1.0, n_leapfrog=10, eps_max=0.3, jump=0, jump_leapfrog=10, jump_eps_max=0.05,
                fixed_bias_index=0, mass_mode=0, seed=0):
    return bps_config(int(n_bins), float(alpha), int(n_leapfrog), float(eps_max), int(jump), int(jump_leapfrog),
                      float(jump_eps_max), int(fixed_bias_index), int(mass_mode), int(seed))


def bps_create(grid_n, box_len, n_sub, cfg, stream=None):
    lib = load()
    ctx = _P()
    st = lib.bps_create(int(grid_n), float(box_len), int(n_sub), ctypes.byref(cfg), _stream_ptr(stream),
                        ctypes.byref(ctx))
    _check(None, st)
    return ctx


def bps_destroy(ctx):
    load().bps_destroy(ctx)


def bps_set_data(ctx, counts, R):
    _check(ctx, load().bps_set_data(ctx, _dptr(counts), _dptr(R)))


def bps_set_data_host(ctx, counts, R):
    c = np.ascontiguousarray(counts, dtype=np.int32)
    r = np.ascontiguousarray(R, dtype=np.float32)
    _check(ctx, load().bps_set_data_host(ctx, c.ctypes.data_as(_P), r.ctypes.data_as(_P)))


def bps_set_data_host_u16(ctx, counts, R):
    c = np.ascontiguousarray(counts, dtype=np.uint16)
    r = np.ascontiguousarray(R, dtype=np.float32)
    _check(ctx, load().bps_set_data_host_u16(ctx, c.ctypes.data_as(_P), r.ctypes.data_as(_P)))


def bps_stage_data_host_u16(ctx, counts, R):
    """Asynchronous upload (see the C declaration).  The arrays are passed without
    conversion, so that the library copies the caller's memory after this call
    returns: uint16 and float32, C-contiguous, and unchanged until the next call
    that uses the data returns (pinned memory for the copies to overlap)."""
    for a, dt in ((counts, np.uint16), (R, np.float32)):
        if not (isinstance(a, np.ndarray) and a.dtype == dt and a.flags.c_contiguous):
            raise TypeError(f"bps_stage_data_host_u16 needs C-contiguous {np.dtype(dt).name} arrays")
    _check(ctx, load().bps_stage_data_host_u16(ctx, counts.ctypes.data_as(_P), R.ctypes.data_as(_P)))


def bps_set_state(ctx, delta, P, b, nbar, iteration=0):
    _, pP = _darr(P)
    _, pb = _darr(b)
    _, pn = _darr(nbar)
    _check(ctx, load().bps_set_state(ctx, _dptr(delta), pP, pb, pn, int(iteration)))


def bps_get_state(ctx, delta=None, n_bins=None, n_sub=None):
    P = np.zeros(n_bins or 64)
    b = np.zeros(n_sub or 16)
    nb = np.zeros(n_sub or 16)
    it = ctypes.c_uint64(0)
    _check(ctx, load().bps_get_state(ctx, _dptr(delta), P.ctypes.data_as(_D), b.ctypes.data_as(_D),
                                     nb.ctypes.data_as(_D), ctypes.byref(it)))
    return P, b, nb, it.value


def bps_get_spectrum(ctx, spec):
    _check(ctx, load().bps_get_spectrum(ctx, _dptr(spec)))


def bps_set_spectrum(ctx, spec):
    _check(ctx, load().bps_set_spectrum(ctx, _dptr(spec)))


def bps_save_chain(ctx):
    """Checkpoint of the chain as bytes (the library's format)."""
    n = ctypes.c_size_t(0)
    _check(ctx, load().bps_save_chain(ctx, None, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(ctx, load().bps_save_chain(ctx, buf, ctypes.byref(n)))
    return buf.raw[:n.value]


def bps_load_chain(ctx, blob):
    b = bytes(blob)
    _check(ctx, load().bps_load_chain(ctx, ctypes.c_char_p(b), len(b)))


def bps_selftest_wait(ctx, limit_ns):
    _check(ctx, load().bps_selftest_wait(ctx, int(limit_ns)))


def bps_mock_field(ctx, seed, P_n2, delta):
    """delta (float32 CUDA tensor [N]^3) <- the true field of Sec. 5 with power P_n2 [3 (N/2)^2 + 1]."""
    a, p = _darr(P_n2)
    _check(ctx, load().bps_mock_field(ctx, int(seed), p, _dptr(delta)))


def bps_mock_counts(ctx, seed, delta, R, b, nbar, noise, counts):
    """counts (int32 CUDA tensor [n_sub][N]^3) <- counts of Eq. data_model; noise 0 Poisson, 1 Gaussian."""
    ab, pb = _darr(b)
    an, pn = _darr(nbar)
    _check(ctx, load().bps_mock_counts(ctx, int(seed), _dptr(delta), _dptr(R), pb, pn, int(noise), _dptr(counts)))


def bps_mock_response(ctx, f_sky, axis, table, R):
    """R (float32 CUDA tensor [n_sub][N]^3) <- cap of sky fraction f_sky about axis x the radial tables."""
    ax, pa = _darr(axis, 3)
    t = np.ascontiguousarray(np.asarray(table, dtype=np.float64))
    _check(ctx, load().bps_mock_response(ctx, float(f_sky), pa, int(t.shape[-1]), t.ctypes.data_as(_D), _dptr(R)))


def bps_schechter_tables(M_edges, r_max, n_r, M_star=-20.44, alpha=-1.05, m_bright=14.5, m_faint=17.77,
                         omega_m=0.24):
    """(table [n_sub][n_r], nbar_rel [n_sub]) of the Schechter selection (host code of the library)."""
    e, pe = _darr(M_edges)
    n_sub = e.size - 1
    sp = bps_schechter(M_star, alpha, m_bright, m_faint, omega_m)
    table = np.zeros((n_sub, int(n_r)))
    nb = np.zeros(n_sub)
    _check(None, load().bps_schechter_tables(ctypes.byref(sp), n_sub, pe, float(r_max), int(n_r),
                                             table.ctypes.data_as(_D), nb.ctypes.data_as(_D)))
    return table, nb


def bps_bias_law(M, b_star=1.2, M_star=-20.83, a=0.895, b=0.105, c=-0.040):
    m, pm = _darr(M)
    out = np.zeros(m.size)
    _check(None, load().bps_bias_law(int(m.size), pm, float(b_star), float(M_star), float(a), float(b), float(c),
                                     out.ctypes.data_as(_D)))
    return out


def bps_posterior_moments(ctx, enable=True):
    _check(ctx, load().bps_posterior_moments(ctx, int(bool(enable))))


def bps_posterior_read(ctx, n_bins, n_sub, mean=None, var=None):
    """(param_mean [D], param_cov [D][D], n); mean / var: optional float64 CUDA tensors [N]^3."""
    D = n_bins + 2 * n_sub
    pm = np.zeros(D)
    pc = np.zeros((D, D))
    n = ctypes.c_uint64(0)
    _check(ctx, load().bps_posterior_read(ctx, _dptr(mean), _dptr(var), pm.ctypes.data_as(_D),
                                          pc.ctypes.data_as(_D), ctypes.byref(n)))
    return pm, pc, n.value


def bps_hmc_step(ctx, want_info=True):
    info = bps_move_info()
    _check(ctx, load().bps_hmc_step(ctx, ctypes.byref(info) if want_info else None))
    return (info.accepted, info.dH, info.eps) if want_info else None


def bps_adapt_step_size(ctx, n_rounds, moves_per_round, target):
    out = np.zeros(1)
    _check(ctx, load().bps_adapt_step_size(ctx, int(n_rounds), int(moves_per_round), float(target),
                                           out.ctypes.data_as(_D)))
    return float(out[0])


def bps_sample_power(ctx, n_bins, want=True):
    if not want:
        _check(ctx, load().bps_sample_power(ctx, None, None))
        return None
    P = np.zeros(n_bins)
    s = np.zeros(n_bins)
    _check(ctx, load().bps_sample_power(ctx, P.ctypes.data_as(_D), s.ctypes.data_as(_D)))
    return P, s


def bps_sample_bias_norm(ctx, n_sub, want=True):
    if not want:
        _check(ctx, load().bps_sample_bias_norm(ctx, None, None, None))
        return None
    b = np.zeros(n_sub)
    nb = np.zeros(n_sub)
    sums = np.zeros(3 * n_sub)
    _check(ctx, load().bps_sample_bias_norm(ctx, b.ctypes.data_as(_D), nb.ctypes.data_as(_D),
                                            sums.ctypes.data_as(_D)))
    return b, nb, sums.reshape(n_sub, 3)


def bps_jump(ctx, want_info=True):
    info = bps_move_info()
    _check(ctx, load().bps_jump(ctx, ctypes.byref(info) if want_info else None))
    return (info.accepted, info.dH, info.eps) if want_info else None


def bps_gibbs_iterate(ctx, n_iter, rec_len=None):
    if rec_len is None:
        _check(ctx, load().bps_gibbs_iterate(ctx, int(n_iter), None))
        return None
    out = np.zeros(int(n_iter) * rec_len)
    _check(ctx, load().bps_gibbs_iterate(ctx, int(n_iter), out.ctypes.data_as(_D)))
    return out.reshape(int(n_iter), rec_len)


def bps_set_mass_scale(ctx, scales):
    a, p = _darr(scales)
    _check(ctx, load().bps_set_mass_scale(ctx, int(a.size), p))


def bps_fft_r2c(ctx, real, spec):
    _check(ctx, load().bps_fft_r2c(ctx, _dptr(real), _dptr(spec)))


def bps_fft_c2r(ctx, spec, real):
    _check(ctx, load().bps_fft_c2r(ctx, _dptr(spec), _dptr(real)))


def bps_gradient(ctx, grad):
    e = np.zeros(2)
    _check(ctx, load().bps_gradient(ctx, _dptr(grad), e.ctypes.data_as(_D)))
    return e


def bps_philox_words(seed, iteration, stage, sub, block0, out, stream=None):
    _check(None, load().bps_philox_words(int(seed), int(iteration), int(stage), int(sub), int(block0),
                                         int(out.numel()), _dptr(out), _stream_ptr(stream)))


def bps_voxel_normals(seed, iteration, out, stream=None):
    _check(None, load().bps_voxel_normals(int(seed), int(iteration), int(out.numel()), _dptr(out),
                                          _stream_ptr(stream)))


def bps_bin_power_noalloc(grid_n, box_len, n_bins, spec, sigma, stream=None):
    """sigma (float64 CUDA tensor [n_bins]) <- k-bin power of spec, no device allocation."""
    _check(None, load().bps_bin_power_noalloc(int(grid_n), float(box_len), int(n_bins), _dptr(spec), _dptr(sigma),
                                              _stream_ptr(stream)))


def bps_create_batch(grid_n, box_len, n_sub, cfg, stream=None):
    lib = load()
    g = np.ascontiguousarray(grid_n, dtype=np.int32)
    bx = np.ascontiguousarray(box_len, dtype=np.float64)
    ns = np.ascontiguousarray(n_sub, dtype=np.int32)
    ctx = _P()
    st = lib.bps_create_batch(int(g.size), g.ctypes.data_as(_P), bx.ctypes.data_as(_P), ns.ctypes.data_as(_P),
                              ctypes.byref(cfg), _stream_ptr(stream), ctypes.byref(ctx))
    _check(None, st)
    return ctx


def bps_batch_set_chain(ctx, chain, counts, R, delta, P, b, nbar, iteration=0):
    _, pP = _darr(P)
    _, pb = _darr(b)
    _, pn = _darr(nbar)
    _check(ctx, load().bps_batch_set_chain(ctx, int(chain), _dptr(counts), _dptr(R), _dptr(delta), pP, pb, pn,
                                           int(iteration)))


def bps_batch_get_chain(ctx, chain, delta=None, n_bins=64, n_sub=16):
    P = np.zeros(n_bins)
    b = np.zeros(n_sub)
    nb = np.zeros(n_sub)
    it = ctypes.c_uint64(0)
    _check(ctx, load().bps_batch_get_chain(ctx, int(chain), _dptr(delta), P.ctypes.data_as(_D),
                                           b.ctypes.data_as(_D), nb.ctypes.data_as(_D), ctypes.byref(it)))
    return P, b, nb, it.value


def bps_batch_record_len(ctx):
    return int(load().bps_batch_record_len(ctx))


def bps_batch_record_slot(ctx, chain):
    return int(load().bps_batch_record_slot(ctx, int(chain)))


def bps_batch_gibbs_iterate(ctx, n_iter, n_chains=None):
    if n_chains is None:
        _check(ctx, load().bps_batch_gibbs_iterate(ctx, int(n_iter), None))
        return None
    rl = bps_batch_record_len(ctx)
    out = np.zeros(int(n_iter) * n_chains * rl)
    _check(ctx, load().bps_batch_gibbs_iterate(ctx, int(n_iter), out.ctypes.data_as(_D)))
    return out.reshape(int(n_iter), n_chains, rl)


class MLP:
    """The mass-preconditioner network (device parameters; FP32 host views)."""

    def __init__(self, sizes, stream=None):
        self.sizes = [int(x) for x in sizes]
        arr = np.ascontiguousarray(self.sizes, dtype=np.int32)
        self.ptr = _P()
        _check(None, load().bps_mlp_create(len(sizes) - 1, arr.ctypes.data_as(_P), _stream_ptr(stream),
                                           ctypes.byref(self.ptr)))
        self.n_params = int(load().bps_mlp_num_params(self.ptr))

    def _chk(self, st):
        _check(None, st)

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.size == self.n_params
        self._chk(load().bps_mlp_set_params(self.ptr, a.ctypes.data_as(_P)))

    def get_params(self):
        a = np.zeros(self.n_params, dtype=np.float32)
        self._chk(load().bps_mlp_get_params(self.ptr, a.ctypes.data_as(_P)))
        return a

    def forward(self, x, y):
        self._chk(load().bps_mlp_forward(self.ptr, int(x.shape[0]), _dptr(x), _dptr(y)))

    def loss_grad(self, x, t):
        loss = ctypes.c_double(0.0)
        g = np.zeros(self.n_params, dtype=np.float32)
        self._chk(load().bps_mlp_loss_grad(self.ptr, int(x.shape[0]), _dptr(x), _dptr(t), ctypes.byref(loss),
                                           g.ctypes.data_as(_P)))
        return loss.value, g

    def adam_step(self, lr):
        self._chk(load().bps_mlp_adam_step(self.ptr, float(lr)))

    def train(self, x, t, batch, steps, lr, seed=0):
        loss = ctypes.c_double(0.0)
        self._chk(load().bps_mlp_train(self.ptr, int(x.shape[0]), _dptr(x), _dptr(t), int(batch), int(steps),
                                       float(lr), int(seed), ctypes.byref(loss)))
        return loss.value

    def close(self):
        if self.ptr is not None:
            load().bps_mlp_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def flatten_params(params):
    """oracle-style [W1, b1, W2, b2, ...] (float64) -> the library's flat FP32 vector."""
    return np.concatenate([np.asarray(p, dtype=np.float32).ravel() for p in params])


def unflatten_params(flat, sizes):
    out, off = [], 0
    for n_in, n_out in zip(sizes[:-1], sizes[1:]):
        out.append(np.asarray(flat[off:off + n_in * n_out], dtype=np.float64).reshape(n_in, n_out))
        off += n_in * n_out
        out.append(np.asarray(flat[off:off + n_out], dtype=np.float64))
        off += n_out
    return out


def bps_mass_stats(ctx, n_moves, n_mass_bins, n_slots=1):
    """(V [n_slots, n_mass], Mbar [n_slots, n_mass]) of the chains' density modes."""
    out = np.zeros(n_slots * 2 * n_mass_bins)
    _check(ctx, load().bps_mass_stats(ctx, int(n_moves), int(n_mass_bins), out.ctypes.data_as(_D)))
    out = out.reshape(n_slots, 2, n_mass_bins)
    return out[:, 0], out[:, 1]


def bps_window_power(ctx, n_bins, n_slots=1):
    out = np.zeros(n_slots * n_bins)
    _check(ctx, load().bps_window_power(ctx, out.ctypes.data_as(_D)))
    return out.reshape(n_slots, n_bins)


def bps_set_mass_net(ctx, net, feat_mean=None, feat_std=None, log_clamp=None):
    """Install `net` (an MLP) as the per-move mass of ctx; net=None removes it."""
    if net is None:
        _check(ctx, load().bps_set_mass_net(ctx, None, None, None, 1.0))
        return
    mu = np.ascontiguousarray(feat_mean, dtype=np.float32)
    sd = np.ascontiguousarray(feat_std, dtype=np.float32)
    _check(ctx, load().bps_set_mass_net(ctx, net.ptr, mu.ctypes.data_as(_P), sd.ctypes.data_as(_P),
                                        float(log_clamp)))


def bps_mlp_export(net, feat_mean, feat_std, log_clamp):
    """The library-format bytes of a trained preconditioner."""
    mu = np.ascontiguousarray(feat_mean, dtype=np.float32)
    sd = np.ascontiguousarray(feat_std, dtype=np.float32)
    n = ctypes.c_size_t(0)
    _check(None, load().bps_mlp_export(net.ptr, mu.ctypes.data_as(_P), sd.ctypes.data_as(_P), float(log_clamp), None,
                                       ctypes.byref(n)))
    buf = (ctypes.c_ubyte * n.value)()
    _check(None, load().bps_mlp_export(net.ptr, mu.ctypes.data_as(_P), sd.ctypes.data_as(_P), float(log_clamp), buf,
                                       ctypes.byref(n)))
    return bytes(buf)


def bps_set_preconditioner(ctx, blob):
    buf = (ctypes.c_ubyte * len(blob)).from_buffer_copy(blob)
    _check(ctx, load().bps_set_preconditioner(ctx, buf, len(blob)))


def bps_get_mass_scale(ctx, chain=0):
    n = ctypes.c_int(0)
    out = np.zeros(64)
    _check(ctx, load().bps_get_mass_scale(ctx, int(chain), ctypes.byref(n), out.ctypes.data_as(_D)))
    return out[:n.value].copy()


def bps_z_line_pairs(ctx):
    return int(load().bps_z_line_pairs(ctx))


def bps_x_pass_variant(ctx):
    return int(load().bps_x_pass_variant(ctx))


def bps_version():
    return load().bps_version().decode()


def bps_kernel_launches(ctx):
    return int(load().bps_kernel_launches(ctx))


def bps_profile(ctx, enable):
    _check(ctx, load().bps_profile(ctx, int(enable)))


def bps_profile_read(ctx):
    ms = np.zeros(4)
    n = (ctypes.c_uint64 * 4)()
    _check(ctx, load().bps_profile_read(ctx, ms.ctypes.data_as(_D), n))
    return ms, np.array(list(n), dtype=np.int64)


class Sampler:
    """One chain of the sampler on the current CUDA device (owns a bps context)."""

    def __init__(self, N, box, n_sub, n_bins, stream=None, **cfg):
        self.N, self.box, self.n_sub, self.n_bins = int(N), float(box), int(n_sub), int(n_bins)
        self.cfg = make_config(n_bins, **cfg)
        self.ctx = bps_create(N, box, n_sub, self.cfg, stream)

    @property
    def rec_len(self):
        return self.n_bins + 2 * self.n_sub + 2

    def close(self):
        if self.ctx is not None:
            bps_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
