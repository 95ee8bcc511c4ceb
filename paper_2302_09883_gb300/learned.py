"""Learned per-patch threshold: features/labels of patches and the small MLP
(C-ABI wrappers; features, labels, training and inference run in the
library's CUDA kernels).  Device arrays are torch CUDA tensors."""
import ctypes as C

import numpy as np

from . import _lib as B

NH = 64


def nparam(nin):
    return NH * nin + NH + NH * NH + NH + NH + 1


def features_labels(dense, P, L, delta, wavelet="bl53", stream=None):
    """dense: CUDA float32 tensor (F, ny, nx), periodic.  Returns CUDA
    tensors (npatch, 6L) float32 features and (npatch,) float32 labels
    (log10 eps)."""
    import torch
    F, ny, nx = dense.shape
    npatch = (nx // P) * (ny // P)
    feat = torch.empty((npatch, 6 * L), dtype=torch.float32, device=dense.device)
    lab = torch.empty((npatch,), dtype=torch.float32, device=dense.device)
    d = dense.contiguous()
    torch.cuda.synchronize()
    st = B.lib().wcs_features_labels(d.data_ptr(), F, nx, ny, B.WAVELET[wavelet], P, L, delta, feat.data_ptr(),
                                     lab.data_ptr(), stream)
    B.check(st, None)
    torch.cuda.synchronize()
    return feat, lab


def features_labels3(dense, P, L, delta, stream=None):
    """dense: CUDA float32 tensor (F, nz, ny, nx), periodic, cubic BL5/3
    patches.  Returns CUDA tensors (npatch, 14L) float32 features and
    (npatch,) float32 labels (log10 eps)."""
    import torch
    F, nz, ny, nx = dense.shape
    npatch = (nx // P) * (ny // P) * (nz // P)
    feat = torch.empty((npatch, 14 * L), dtype=torch.float32, device=dense.device)
    lab = torch.empty((npatch,), dtype=torch.float32, device=dense.device)
    d = dense.contiguous()
    torch.cuda.synchronize()
    st = B.lib().wcs_features_labels3(d.data_ptr(), F, nx, ny, nz, P, L, delta, feat.data_ptr(), lab.data_ptr(), stream)
    B.check(st, None)
    torch.cuda.synchronize()
    return feat, lab


class Mlp:
    def __init__(self, nin, weights=None, seed=0):
        h = C.c_void_p()
        B.check(B.lib().wcs_mlp_create(nin, C.byref(h)), None)
        self.h, self.nin = h, nin
        if weights is None:
            rng = np.random.default_rng(seed)
            w = np.zeros(nparam(nin), np.float32)
            o = 0
            for fan_in, fan_out in [(nin, NH), (NH, NH), (NH, 1)]:
                w[o:o + fan_in * fan_out] = rng.normal(0, 1 / np.sqrt(fan_in), fan_in * fan_out)
                o += fan_in * fan_out + fan_out
            weights = w
        self.set_weights(weights)

    def close(self):
        if getattr(self, "h", None):
            B.lib().wcs_mlp_destroy(self.h)
            self.h = None

    __del__ = close

    def set_weights(self, w):
        w = np.ascontiguousarray(w, np.float32)
        B.check(B.lib().wcs_mlp_set_weights(self.h, w.ctypes.data_as(C.POINTER(C.c_float))), None)

    def weights(self):
        w = np.zeros(nparam(self.nin), np.float32)
        B.check(B.lib().wcs_mlp_get_weights(self.h, w.ctypes.data_as(C.POINTER(C.c_float))), None)
        return w

    def grad(self, X, t):
        import torch
        X, t = X.float().contiguous(), t.float().contiguous()
        torch.cuda.synchronize()
        g = np.zeros(nparam(self.nin), np.float32)
        loss = C.c_float()
        B.check(B.lib().wcs_mlp_grad(self.h, X.data_ptr(), t.data_ptr(), X.shape[0],
                                     g.ctypes.data_as(C.POINTER(C.c_float)), C.byref(loss)), None)
        return float(loss.value), g

    def train(self, X, t, epochs, batch, lr, seed=0):
        import torch
        X, t = X.float().contiguous(), t.float().contiguous()
        torch.cuda.synchronize()
        n = X.shape[0]
        nb = n // batch
        rng = np.random.default_rng(seed)
        idx = np.concatenate([rng.permutation(n)[:nb * batch] for _ in range(epochs)]).astype(np.int32)
        hist = np.zeros(epochs, np.float32)
        B.check(B.lib().wcs_mlp_train(self.h, X.data_ptr(), t.data_ptr(), n, idx.ctypes.data_as(C.POINTER(C.c_int)),
                                      epochs, batch, lr, hist.ctypes.data_as(C.POINTER(C.c_float))), None)
        return hist

    def forward(self, X):
        import torch
        X = X.float().contiguous()
        y = torch.empty((X.shape[0],), dtype=torch.float32, device=X.device)
        torch.cuda.synchronize()
        B.check(B.lib().wcs_mlp_forward(self.h, X.data_ptr(), X.shape[0], y.data_ptr()), None)
        torch.cuda.synchronize()
        return y


def use_mlp(sim, mlp, eps_lo=1e-7, eps_hi=1e-2):
    B.check(B.lib().wcs_sim_use_mlp(sim.h, mlp.h if mlp is not None else None, eps_lo, eps_hi), sim.h)


def set_patch_eps(sim, eps):
    e = np.ascontiguousarray(eps, np.float64)
    B.check(B.lib().wcs_sim_set_patch_eps(sim.h, e.ctypes.data_as(C.POINTER(C.c_double))), sim.h)


def patch_data(sim, L):
    dims = 3 if len(sim.G) == 3 else 2
    feat = np.zeros((sim.npatch, 2 * ((1 << dims) - 1) * L), np.float32)
    eps = np.zeros(sim.npatch, np.float64)
    B.check(B.lib().wcs_sim_patch_data(sim.h, feat.ctypes.data_as(C.POINTER(C.c_float)),
                                       eps.ctypes.data_as(C.POINTER(C.c_double))), sim.h)
    return feat, eps


def fit(X, t, epochs=200, batch=128, lr=2e-3, seed=0, sd_floor=1e-3):
    """Trains a network on raw features X (CUDA tensor (n, nin)) and targets
    t (log10 eps) in one library call: the library standardises the inputs
    for training and folds the standardisation into the first layer, so the
    returned network takes the raw features that a learned-mode step
    writes.  Only the minibatch permutations are drawn here (seeded).
    Returns (Mlp, loss history)."""
    import torch
    X, t = X.float().contiguous(), t.float().contiguous()
    torch.cuda.synchronize()
    n, nin = X.shape
    m = Mlp(nin, seed=seed)
    nb = n // batch
    rng = np.random.default_rng(seed)
    idx = np.concatenate([rng.permutation(n)[:nb * batch] for _ in range(epochs)]).astype(np.int32)
    hist = np.zeros(epochs, np.float32)
    stats = np.zeros(2 * (nin + 1), np.float64)
    B.check(B.lib().wcs_mlp_fit(m.h, X.data_ptr(), t.data_ptr(), n, idx.ctypes.data_as(C.POINTER(C.c_int)), epochs,
                                batch, lr, sd_floor, hist.ctypes.data_as(C.POINTER(C.c_float)),
                                stats.ctypes.data_as(C.POINTER(C.c_double))), None)
    m.input_stats = stats.reshape(nin + 1, 2)  # (mean, deviation) per input, then of t
    return m, hist
