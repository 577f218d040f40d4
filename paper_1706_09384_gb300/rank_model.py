"""Rank predictor: parameter initialisation, GPU training over builds, I/O.

The model itself (features, network, training and inference kernels) lives
in the CUDA library (see include/hm.h, HM_RANK_MODEL_PARAMS); this module only
draws the seeded initial weights, gathers training samples from H-matrices
built by the library, and calls the library's training kernels.
"""
import os

import numpy as np

from . import hm

NF, NH = 6, 64
HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "rank_model.npy")


def init_params(seed=0):
    """Seeded initial weights (Glorot-uniform layers, zero biases); the first 14
    entries (standardisation constants) are filled in by training."""
    rng = np.random.default_rng(seed)
    P = np.zeros(hm.HM_RANK_MODEL_PARAMS, np.float32)
    P[6:12] = 1.0
    P[13] = 1.0
    o = 14

    def glorot(n_out, n_in):
        a = np.sqrt(6.0 / (n_in + n_out))
        return rng.uniform(-a, a, (n_out, n_in)).astype(np.float32)

    P[o:o + NH * NF] = glorot(NH, NF).ravel()
    o += NH * NF + NH
    P[o:o + NH * NH] = glorot(NH, NH).ravel()
    o += NH * NH + NH
    P[o:o + NH] = glorot(1, NH).ravel()
    return P


def train(feats, targets, steps=3000, batch=2048, lr=2e-3, seed=0, params=None):
    """Trains on the GPU with the library's kernels.  Returns (params, losses)."""
    import torch
    P = init_params(seed) if params is None else np.asarray(params, np.float32).copy()
    dF = torch.from_numpy(np.ascontiguousarray(feats, np.float32)).cuda()
    dT = torch.from_numpy(np.ascontiguousarray(targets, np.float32)).cuda()
    dP = torch.from_numpy(P).cuda()
    losses = np.zeros(steps, np.float32)
    hm._check(hm.lib().hm_rank_model_train(dF.data_ptr(), dT.data_ptr(), len(targets), steps,
                                           batch, lr, seed, dP.data_ptr(),
                                           losses.ctypes.data_as(hm.C.c_void_p),
                                           hm._stream_ptr(None)), "hm_rank_model_train")
    return dP.cpu().numpy(), losses


def predict(params, feats):
    import torch
    dP = torch.from_numpy(np.ascontiguousarray(params, np.float32)).cuda()
    dF = torch.from_numpy(np.ascontiguousarray(feats, np.float32)).cuda()
    out = torch.empty(len(feats), dtype=torch.float32, device="cuda")
    hm._check(hm.lib().hm_rank_model_predict(dP.data_ptr(), dF.data_ptr(), len(feats),
                                             out.data_ptr(), hm._stream_ptr(None)),
              "hm_rank_model_predict")
    return out.cpu().numpy()


def grad(params, feats, targets):
    import torch
    dP = torch.from_numpy(np.ascontiguousarray(params, np.float32)).cuda()
    dF = torch.from_numpy(np.ascontiguousarray(feats, np.float32)).cuda()
    dT = torch.from_numpy(np.ascontiguousarray(targets, np.float32)).cuda()
    g = torch.empty(hm.HM_RANK_MODEL_PARAMS - 14, dtype=torch.float32, device="cuda")
    loss = hm.C.c_float(0.0)
    hm._check(hm.lib().hm_rank_model_grad(dP.data_ptr(), dF.data_ptr(), dT.data_ptr(),
                                          len(targets), g.data_ptr(), hm.C.byref(loss),
                                          hm._stream_ptr(None)), "hm_rank_model_grad")
    return loss.value, g.cpu().numpy()


def load(path=DEFAULT_WEIGHTS):
    return np.load(path).astype(np.float32)
