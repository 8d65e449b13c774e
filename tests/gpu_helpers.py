"""Shared helpers of the GPU parity tests: inputs from the seeded generator, oracle references
and the comparison metrics (stated tolerances are in the tests)."""
import os

import numpy as np

from tests.conftest import ROOT


def torch_dev():
    import torch
    return torch.device("cuda:0")


def gpu_mech(path, **kw):
    from paper_2205_05681_gb300 import chem
    return chem.Mechanism(path, **kw)


def to_dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=torch_dev())


def gross_f(om, y, P):
    """Gross magnitude of every f component of one cell: V sum_r |nu_kr| (qf_r + qr_r) for the
    species rows and T sum_k |h_k/RT| (that) / cpm for the temperature row."""
    r = om.rates(y, P)
    n = om.moles_all(y)[0]
    V = n.sum() * 8314.462618 * y[0] / P
    g_sp = V * (np.abs(om.nu_r - om.nu_f).T @ (r["qf"] + r["qr"]))
    th = np.array([om.thermo(k, y[0]) for k in range(om.ns)])
    cpm = (n * th[:, 0]).sum()
    gT = y[0] * (np.abs(th[:, 1]) * g_sp).sum() / cpm
    return np.concatenate([[gT], g_sp[:-1]])


def weighted_norm(y_ref, y, rtol=1e-6, atol=1e-10):
    """Per-cell RMS of |y_ref - y| / (atol + rtol |y_ref|) (Eq. e:ivp_norm in RMS form)."""
    w = atol + rtol * np.abs(y_ref)
    return np.sqrt(np.mean(((y - y_ref) / w) ** 2, axis=1))


def gpu_state(om, T, Y):
    """oracle-layout state y[c, :] from GPU T [C] and Y [Ns, C] tensors"""
    return om.state_from_TY(T.cpu().numpy(), Y.cpu().numpy().T)
