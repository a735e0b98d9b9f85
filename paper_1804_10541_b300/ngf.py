"""Thin ctypes binding of the C ABI in include/ngf.h (libngf_b300.so).

Argument marshalling only: every operator runs in the library's CUDA kernels
for sm_103a.  Importing this module loads the in-tree library and raises if it
is missing; there is no other code path.  Functions carry the ABI's names;
tensors are passed as torch CUDA tensors (float32, contiguous) or as raw
integer device pointers, streams as torch.cuda.Stream, raw cudaStream_t
integers or None (the legacy default stream).
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libngf_b300.so")

NGF_OK = 0
STATUS = {0: "NGF_OK", -1: "NGF_EINVAL", -2: "NGF_ECUDA", -3: "NGF_ENOMEM", -4: "NGF_ENONFINITE",
          -5: "NGF_EBREAKDOWN", -6: "NGF_ELINESEARCH", -7: "NGF_EMAXITER", -8: "NGF_EBOUNDS"}
NGF_PCG_NSCALARS = 8

# every function include/ngf.h declares
EXPORTS = ["ngf_plan_create", "ngf_plan_destroy", "ngf_plan_set_stream", "ngf_last_error", "ngf_objective",
           "ngf_objective_dev", "ngf_gradient", "ngf_gradient_dev", "gn_hessvec", "curvature_apply",
           "ngf_gn_diagonal", "pcg_init", "pcg_step", "pcg_solve", "pcg_read", "register_multilevel",
           "ngf_objective_noalloc", "ngf_profile_enable", "ngf_profile_read", "ngf_launch_count",
           "ngf_batch_create", "ngf_batch_destroy", "ngf_batch_objective", "ngf_batch_gradient",
           "ngf_batch_hessvec", "ngf_batch_diagonal", "ngf_batch_autotune", "ngf_batch_zc", "register_batch",
           "ngf_h0_solve", "ngf_plan_create_ex", "ngf_conv3d_fwd", "ngf_conv3d_check", "ngf_conv3d_fwd_ex",
           "ngf_conv3d_dgrad", "ngf_conv3d_wgrad", "ngf_net_param_count", "ngf_net_create", "ngf_net_destroy",
           "ngf_net_set_params", "ngf_net_get_params", "ngf_net_forward", "ngf_net_grad", "ngf_net_train_step",
           "ngf_net_train"]
NGF_METHOD_GN, NGF_METHOD_LBFGS = 0, 1


NGF_DIST_NGF, NGF_DIST_SSD = 0, 1


class LevelDesc(C.Structure):
    _fields_ = [("m", C.c_int32 * 3), ("h", C.c_double * 3), ("n", C.c_int32 * 3),
                ("alpha", C.c_double), ("tau", C.c_double), ("rho", C.c_double), ("distance", C.c_int32)]


class PcgState(C.Structure):
    _fields_ = [("x", C.c_void_p), ("r", C.c_void_p), ("z", C.c_void_p), ("d", C.c_void_p),
                ("q", C.c_void_p), ("diag", C.c_void_p), ("dev_scalars", C.c_void_p), ("rtol", C.c_double)]


class PcgInfo(C.Structure):
    _fields_ = [("iters_done", C.c_int32), ("status", C.c_int32), ("delta", C.c_double), ("rr", C.c_double)]


class Options(C.Structure):
    _fields_ = [("levels", C.c_int32), ("gn_iters", C.c_int32), ("pcg_iters", C.c_int32), ("ls_max", C.c_int32),
                ("armijo_c1", C.c_double), ("pcg_rtol", C.c_double), ("start_level", C.c_int32),
                ("u_init", C.c_void_p), ("use_graph", C.c_int32), ("method", C.c_int32),
                ("lbfgs_memory", C.c_int32), ("lbfgs_gamma", C.c_double), ("zc", C.c_int32),
                ("gn_iters_finest", C.c_int32), ("j_target", C.c_double), ("diag_every", C.c_int32)]


class Report(C.Structure):
    _fields_ = [("J", C.c_double), ("D", C.c_double), ("S", C.c_double), ("gn_done", C.c_int32),
                ("pcg_total", C.c_int32), ("ls_trials", C.c_int32), ("ls_fail", C.c_int32),
                ("status", C.c_int32), ("seconds", C.c_double), ("hessvec_voxels", C.c_int64)]


class NetDesc(C.Structure):
    _fields_ = [("s", C.c_int32), ("max_batch", C.c_int32), ("in_shift", C.c_float), ("in_scale", C.c_float),
                ("out_scale", C.c_float)]


class NGFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def declare(lib):
    """Attach argument/return types of every exported function to `lib`."""
    P, D, I32, VP = C.c_void_p, C.POINTER(C.c_double), C.c_int32, C.c_void_p
    sig = {
        "ngf_plan_create": [C.POINTER(C.c_void_p), C.POINTER(LevelDesc), VP],
        "ngf_plan_destroy": [P],
        "ngf_plan_set_stream": [P, VP],
        "ngf_objective": [P, VP, VP, VP, D, D],
        "ngf_objective_dev": [P, VP, VP, VP, VP],
        "ngf_gradient": [P, VP, VP, VP, VP, D, D],
        "ngf_gradient_dev": [P, VP, VP, VP, VP, VP],
        "gn_hessvec": [P, VP, VP, VP, VP, VP],
        "curvature_apply": [P, VP, VP, D],
        "ngf_gn_diagonal": [P, VP, VP, VP, VP],
        "pcg_init": [P, C.POINTER(PcgState), VP],
        "pcg_step": [P, C.POINTER(PcgState), VP, VP, VP],
        "pcg_solve": [P, C.POINTER(PcgState), VP, VP, VP, I32, I32],
        "pcg_read": [P, C.POINTER(PcgState), C.POINTER(PcgInfo)],
        "register_multilevel": [C.POINTER(LevelDesc), C.POINTER(Options), VP, VP, VP, C.POINTER(Report), VP],
        "ngf_objective_noalloc": [C.POINTER(LevelDesc), VP, VP, VP, VP, VP],
        "ngf_profile_enable": [P, I32],
        "ngf_profile_read": [P, I32, D, C.POINTER(C.c_int64)],
        "ngf_batch_create": [C.POINTER(C.c_void_p), I32, C.POINTER(LevelDesc), I32, VP],
        "ngf_batch_destroy": [P],
        "ngf_batch_objective": [P, VP, VP, VP, D, D],
        "ngf_batch_gradient": [P, VP, VP, VP, VP],
        "ngf_batch_hessvec": [P, VP, VP, VP, VP, VP],
        "ngf_batch_diagonal": [P, VP, VP, VP, VP],
        "ngf_batch_autotune": [P, VP, VP, VP, VP, VP, C.POINTER(I32), D],
        "register_batch": [I32, C.POINTER(LevelDesc), C.POINTER(Options), VP, VP, VP, C.POINTER(Report), I32, VP],
        "ngf_h0_solve": [P, C.c_double, VP, VP],
        "ngf_plan_create_ex": [C.POINTER(C.c_void_p), C.POINTER(LevelDesc), I32, VP],
        "ngf_conv3d_fwd": [VP, VP, VP, VP, I32, I32, I32, I32, I32, I32, I32, VP],
        "ngf_conv3d_check": [VP],
        "ngf_conv3d_fwd_ex": [VP, VP, VP, VP, I32, I32, I32, I32, I32, I32, I32, VP],
        "ngf_conv3d_dgrad": [VP, VP, VP, I32, I32, I32, I32, I32, I32, I32, VP],
        "ngf_conv3d_wgrad": [VP, VP, VP, VP, I32, I32, I32, I32, I32, I32, VP],
        "ngf_net_create": [C.POINTER(C.c_void_p), C.POINTER(NetDesc), VP],
        "ngf_net_destroy": [P],
        "ngf_net_set_params": [P, VP],
        "ngf_net_get_params": [P, VP],
        "ngf_net_forward": [P, VP, VP, I32, VP],
        "ngf_net_grad": [P, VP, VP, VP, I32, VP, D],
        "ngf_net_train_step": [P, VP, VP, VP, I32, C.c_double, D],
        "ngf_net_train": [P, VP, VP, VP, I32, C.POINTER(I32), I32, I32, C.c_double, D],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.ngf_last_error.argtypes = [P]
    lib.ngf_last_error.restype = C.c_char_p
    lib.ngf_launch_count.argtypes = []
    lib.ngf_launch_count.restype = C.c_int64
    lib.ngf_net_param_count.argtypes = [C.POINTER(NetDesc)]
    lib.ngf_net_param_count.restype = C.c_int64
    lib.ngf_batch_zc.argtypes = [P]
    lib.ngf_batch_zc.restype = C.c_int32
    return lib


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libngf_b300.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    return declare(C.CDLL(LIB_PATH))


lib = _load()


def _check(status, plan=None):
    if status != NGF_OK:
        raise NGFError(status, lib.ngf_last_error(plan).decode())


def _ptr(x):
    """Device (or host) address of a tensor / array / integer pointer."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def level_desc(m, h, n, alpha=1.0, tau=0.1, rho=0.1, distance=NGF_DIST_NGF):
    d = LevelDesc()
    d.distance = int(distance)
    for a in range(3):
        d.m[a], d.h[a], d.n[a] = int(m[a]), float(h[a]), int(n[a])
    d.alpha, d.tau, d.rho = float(alpha), float(tau), float(rho)
    return d


# ---- same-name wrappers of the C ABI ---------------------------------------

def ngf_plan_create(desc, stream=None):
    h = C.c_void_p()
    _check(lib.ngf_plan_create(C.byref(h), C.byref(desc), _stream(stream)))
    return h


def ngf_plan_create_ex(desc, zc, stream=None):
    h = C.c_void_p()
    _check(lib.ngf_plan_create_ex(C.byref(h), C.byref(desc), int(zc), _stream(stream)))
    return h


def ngf_conv3d_fwd(x, w, bias, y, relu=False, stream=None):
    """3x3x3 convolution on the tensor cores: x [B][D][H][W][Cin] bf16,
    w [Cout][3][3][3][Cin] bf16, bias [Cout] float or None, y
    [B][D][H][W][Cout] float (all device, contiguous)."""
    B, D, H, W, Cin = x.shape
    Cout = w.shape[0]
    _check(lib.ngf_conv3d_fwd(_ptr(x), _ptr(w), _ptr(bias) if bias is not None else None, _ptr(y),
                              B, D, H, W, Cin, Cout, 1 if relu else 0, _stream(stream)))


NGF_CONV_RELU, NGF_CONV_OUT_BF16 = 1, 2


def ngf_conv3d_fwd_ex(x, w, bias, y, flags=0, stream=None):
    """3x3x3 convolution with flags (NGF_CONV_RELU, NGF_CONV_OUT_BF16): y is
    float, or bf16 with NGF_CONV_OUT_BF16."""
    B, D, H, W, Cin = x.shape
    Cout = w.shape[0]
    _check(lib.ngf_conv3d_fwd_ex(_ptr(x), _ptr(w), _ptr(bias) if bias is not None else None, _ptr(y),
                                 B, D, H, W, Cin, Cout, int(flags), _stream(stream)))


def ngf_conv3d_dgrad(dy, w, dx, flags=0, stream=None):
    """Data gradient of a layer with weights w [Cout][3][3][3][Cin]: dy
    [B][D][H][W][Cout] bf16 -> dx [B][D][H][W][Cin] float (bf16 with
    NGF_CONV_OUT_BF16)."""
    B, D, H, W, Cout = dy.shape
    Cin = w.shape[4]
    _check(lib.ngf_conv3d_dgrad(_ptr(dy), _ptr(w), _ptr(dx), B, D, H, W, Cin, Cout, int(flags), _stream(stream)))


def ngf_conv3d_wgrad(dy, x, dw, db=None, stream=None):
    """Weight (and bias) gradient: dy [..][Cout] bf16, x [..][Cin] bf16 ->
    dw [Cout][3][3][3][Cin] float, db [Cout] float (optional)."""
    B, D, H, W, Cin = x.shape
    Cout = dy.shape[4]
    _check(lib.ngf_conv3d_wgrad(_ptr(dy), _ptr(x), _ptr(dw), _ptr(db) if db is not None else None,
                                B, D, H, W, Cin, Cout, _stream(stream)))


def ngf_conv3d_check(stream=None):
    """Number of convolution waits that gave up since the last call."""
    n = lib.ngf_conv3d_check(_stream(stream))
    if n < 0:
        _check(n)
    return n


def ngf_plan_destroy(plan):
    _check(lib.ngf_plan_destroy(plan))


def ngf_plan_set_stream(plan, stream):
    _check(lib.ngf_plan_set_stream(plan, _stream(stream)), plan)


def ngf_last_error(plan=None):
    return lib.ngf_last_error(plan).decode()


def ngf_objective(plan, R, T, u):
    D, S = C.c_double(), C.c_double()
    _check(lib.ngf_objective(plan, _ptr(R), _ptr(T), _ptr(u), C.byref(D), C.byref(S)), plan)
    return D.value, S.value


def ngf_objective_dev(plan, R, T, u, dev_DS):
    _check(lib.ngf_objective_dev(plan, _ptr(R), _ptr(T), _ptr(u), _ptr(dev_DS)), plan)


def ngf_objective_noalloc(desc, R, T, u, dev_DS, stream=None):
    """D, S into dev_DS (device, 2 doubles) without a plan and without any
    device allocation (see include/ngf.h for who needs this and its limits)."""
    _check(lib.ngf_objective_noalloc(C.byref(desc), _ptr(R), _ptr(T), _ptr(u), _ptr(dev_DS), _stream(stream)))


def ngf_gradient(plan, R, T, u, grad, want_scalars=True):
    if not want_scalars:
        _check(lib.ngf_gradient(plan, _ptr(R), _ptr(T), _ptr(u), _ptr(grad), None, None), plan)
        return None
    D, S = C.c_double(), C.c_double()
    _check(lib.ngf_gradient(plan, _ptr(R), _ptr(T), _ptr(u), _ptr(grad), C.byref(D), C.byref(S)), plan)
    return D.value, S.value


def ngf_gradient_dev(plan, R, T, u, grad, dev_DS=None):
    _check(lib.ngf_gradient_dev(plan, _ptr(R), _ptr(T), _ptr(u), _ptr(grad), _ptr(dev_DS)), plan)


def gn_hessvec(plan, R, T, u, p, q):
    _check(lib.gn_hessvec(plan, _ptr(R), _ptr(T), _ptr(u), _ptr(p), _ptr(q)), plan)


def curvature_apply(plan, p, q=None, want_S=True):
    Sp = C.c_double()
    _check(lib.curvature_apply(plan, _ptr(p), _ptr(q), C.byref(Sp) if want_S else None), plan)
    return Sp.value if want_S else None


def ngf_gn_diagonal(plan, R, T, u, diag):
    _check(lib.ngf_gn_diagonal(plan, _ptr(R), _ptr(T), _ptr(u), _ptr(diag)), plan)


def pcg_state(x, r, z, d, q, diag, dev_scalars, rtol=0.0):
    st = PcgState()
    st.x, st.r, st.z, st.d, st.q = _ptr(x), _ptr(r), _ptr(z), _ptr(d), _ptr(q)
    st.diag, st.dev_scalars, st.rtol = _ptr(diag), _ptr(dev_scalars), float(rtol)
    return st


def pcg_init(plan, st, rhs):
    _check(lib.pcg_init(plan, C.byref(st), _ptr(rhs)), plan)


def pcg_step(plan, st, R, T, u):
    _check(lib.pcg_step(plan, C.byref(st), _ptr(R), _ptr(T), _ptr(u)), plan)


def pcg_solve(plan, st, R, T, u, iters, use_graph=True):
    _check(lib.pcg_solve(plan, C.byref(st), _ptr(R), _ptr(T), _ptr(u), int(iters), 1 if use_graph else 0), plan)


def pcg_read(plan, st):
    info = PcgInfo()
    _check(lib.pcg_read(plan, C.byref(st), C.byref(info)), plan)
    return info


def options(levels, gn_iters=10, pcg_iters=20, ls_max=10, armijo_c1=1e-4, pcg_rtol=0.0, u_init=None,
            start_level=0, use_graph=True, method=NGF_METHOD_GN, lbfgs_memory=5, lbfgs_gamma=0.0, zc=0,
            gn_iters_finest=0, j_target=0.0, diag_every=0):
    o = Options()
    o.levels, o.gn_iters, o.pcg_iters, o.ls_max = levels, gn_iters, pcg_iters, ls_max
    o.armijo_c1, o.pcg_rtol, o.start_level = armijo_c1, pcg_rtol, start_level
    o.u_init = _ptr(u_init)
    o.use_graph = 1 if use_graph else 0
    o.method, o.lbfgs_memory, o.lbfgs_gamma = int(method), int(lbfgs_memory), float(lbfgs_gamma)
    o.zc = int(zc)
    o.gn_iters_finest, o.j_target = int(gn_iters_finest), float(j_target)
    o.diag_every = int(diag_every)
    return o


def ngf_h0_solve(plan, gamma, q, r):
    """r = (alpha grad^2 S + gamma I)^{-1} q (the L-BFGS initial Hessian)."""
    _check(lib.ngf_h0_solve(plan, float(gamma), _ptr(q), _ptr(r)), plan)


def register_multilevel(desc, opts, R, T, u_out, stream=None):
    rep = Report()
    _check(lib.register_multilevel(C.byref(desc), C.byref(opts), _ptr(R), _ptr(T), _ptr(u_out), C.byref(rep),
                                   _stream(stream)))
    return rep


NGF_K_OBJECTIVE, NGF_K_GRADIENT, NGF_K_HESSVEC, NGF_K_DIAGONAL = 0, 1, 2, 3


def ngf_profile_enable(plan, enable=True):
    _check(lib.ngf_profile_enable(plan, 1 if enable else 0), plan)


def ngf_profile_read(plan, which):
    ms, n = C.c_double(), C.c_int64()
    _check(lib.ngf_profile_read(plan, int(which), C.byref(ms), C.byref(n)), plan)
    return ms.value, n.value


def ngf_launch_count():
    return int(lib.ngf_launch_count())


# ---- batched form -----------------------------------------------------------

def _ptr_array(xs):
    """Host array of device pointers (kept alive by the caller's reference)."""
    arr = (C.c_void_p * len(xs))(*[_ptr(x) for x in xs])
    return arr


def ngf_batch_create(descs, zc=0, stream=None):
    arr = (LevelDesc * len(descs))(*descs)
    h = C.c_void_p()
    _check(lib.ngf_batch_create(C.byref(h), len(descs), arr, int(zc), _stream(stream)))
    return h


def ngf_batch_destroy(batch):
    _check(lib.ngf_batch_destroy(batch))


def ngf_batch_zc(batch):
    return int(lib.ngf_batch_zc(batch))


def ngf_batch_objective(batch, R, T, u):
    n = len(R)
    D, S = (C.c_double * n)(), (C.c_double * n)()
    _check(lib.ngf_batch_objective(batch, _ptr_array(R), _ptr_array(T), _ptr_array(u), D, S))
    return list(D), list(S)


def ngf_batch_gradient(batch, R, T, u, grad):
    _check(lib.ngf_batch_gradient(batch, _ptr_array(R), _ptr_array(T), _ptr_array(u), _ptr_array(grad)))


def ngf_batch_hessvec(batch, R, T, u, p, q):
    _check(lib.ngf_batch_hessvec(batch, _ptr_array(R), _ptr_array(T), _ptr_array(u), _ptr_array(p),
                                 _ptr_array(q)))


def ngf_batch_diagonal(batch, R, T, u, diag):
    _check(lib.ngf_batch_diagonal(batch, _ptr_array(R), _ptr_array(T), _ptr_array(u), _ptr_array(diag)))


def ngf_batch_autotune(batch, R, T, u, p, q):
    zc, ms = C.c_int32(), C.c_double()
    _check(lib.ngf_batch_autotune(batch, _ptr_array(R), _ptr_array(T), _ptr_array(u), _ptr_array(p),
                                  _ptr_array(q), C.byref(zc), C.byref(ms)))
    return zc.value, ms.value


def register_batch(descs, opts, R, T, u_out, autotune=False, stream=None):
    n = len(descs)
    reps = (Report * n)()
    _check(lib.register_batch(n, (LevelDesc * n)(*descs), C.byref(opts), _ptr_array(R), _ptr_array(T),
                              _ptr_array(u_out), reps, 1 if autotune else 0, _stream(stream)))
    return list(reps)


class Batch:
    """Owning wrapper of an ngf_batch."""

    def __init__(self, descs, zc=0, stream=None):
        self.descs = list(descs)
        self.handle = ngf_batch_create(self.descs, zc, stream)

    def close(self):
        if self.handle:
            ngf_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Plan:
    """Owning wrapper of an ngf_plan."""

    def __init__(self, desc, stream=None, zc=0):
        self.desc = desc
        self.handle = ngf_plan_create_ex(desc, zc, stream) if zc else ngf_plan_create(desc, stream)

    def close(self):
        if self.handle:
            ngf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ---- learned initializer (encoder-decoder network) ---------------------------

def net_desc(s, max_batch, in_shift, in_scale, out_scale):
    d = NetDesc()
    d.s, d.max_batch = int(s), int(max_batch)
    d.in_shift, d.in_scale, d.out_scale = float(in_shift), float(in_scale), float(out_scale)
    return d


def ngf_net_param_count(desc):
    n = int(lib.ngf_net_param_count(C.byref(desc)))
    if n < 0:
        raise NGFError(-1, "bad network descriptor")
    return n


def ngf_net_create(desc, stream=None):
    h = C.c_void_p()
    _check(lib.ngf_net_create(C.byref(h), C.byref(desc), _stream(stream)))
    return h


def ngf_net_destroy(net):
    _check(lib.ngf_net_destroy(net))


def ngf_net_set_params(net, params):
    _check(lib.ngf_net_set_params(net, _ptr(params)))


def ngf_net_get_params(net, params):
    _check(lib.ngf_net_get_params(net, _ptr(params)))


def ngf_net_forward(net, R, T, B, u):
    _check(lib.ngf_net_forward(net, _ptr(R), _ptr(T), int(B), _ptr(u)))


def ngf_net_grad(net, R, T, u_target, B, grads=None):
    loss = C.c_double()
    _check(lib.ngf_net_grad(net, _ptr(R), _ptr(T), _ptr(u_target), int(B), _ptr(grads), C.byref(loss)))
    return loss.value


def ngf_net_train_step(net, R, T, u_target, B, lr, want_loss=True):
    loss = C.c_double()
    _check(lib.ngf_net_train_step(net, _ptr(R), _ptr(T), _ptr(u_target), int(B), float(lr),
                                  C.byref(loss) if want_loss else None))
    return loss.value if want_loss else None


def ngf_net_train(net, R, T, u_target, npairs, order, batch, lr):
    """Adam steps over the pairs in `order` (batches of `batch`); returns the
    per-batch losses."""
    order = [int(k) for k in order]
    arr = (C.c_int32 * max(1, len(order)))(*order)
    nb = (len(order) + batch - 1) // batch
    losses = (C.c_double * max(1, nb))()
    _check(lib.ngf_net_train(net, _ptr(R), _ptr(T), _ptr(u_target), int(npairs), arr, len(order), int(batch),
                             float(lr), losses))
    return list(losses)[:nb]


class Net:
    """Owning wrapper of an ngf_net."""

    def __init__(self, desc, stream=None):
        self.desc = desc
        self.handle = ngf_net_create(desc, stream)
        self.nparams = ngf_net_param_count(desc)

    def close(self):
        if self.handle:
            ngf_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
