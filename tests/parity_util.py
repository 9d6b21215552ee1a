"""Shared helpers of the GPU parity tests (inputs from workloads, expected
values from the FP64 oracle only)."""
import numpy as np
import torch

import oracle
from paper_2104_00794_gb300 import api


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def problem(w, nt=None, form="levels"):
    return api.Problem.from_workload(w, nt=nt, form=form)


def oracle_dobs(w, nt=None):
    """Observed data from the oracle's FP64 forward on the true model,
    rounded to float32 (the precision both sides then read)."""
    return oracle.batch_forward(w, w.vel_true, nt).astype(np.float32)


def to_dev(a):
    return torch.as_tensor(np.array(a, copy=True, order="C"), device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()
