"""Helpers of the GPU parity tests: seeded inputs on the device, the same
inputs for the oracle in float64, and relative error measures."""
import numpy as np
import torch

from paper_1804_10541_b300 import ngf, synth

# Tolerances of the parity tests (relative L2 unless stated).  The gradient,
# Hessian-vector and objective bars are the stated targets of the GPU path;
# the diagonal shares the Hessian's; PCG iterates amplify the float32
# rounding of each Hessian-vector product by the conditioning of the Krylov
# recursion, hence the looser bar after k iterations.
TOL_GRAD = 1e-5
TOL_HESS = 1e-5
TOL_DIAG = 1e-5
TOL_OBJ = 1e-6   # relative, scalar
TOL_CURV = 1e-5
TOL_PCG = 1e-4


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def f64(t):
    return t.detach().double().cpu().numpy().ravel()


class Case:
    """Device tensors and an oracle level for one (R, T, u, p) problem."""

    def __init__(self, m, h, n, alpha, tau, rho, R, T, u, p, dev="cuda"):
        import oracle as O
        self.m, self.h, self.n = tuple(m), tuple(h), tuple(n)
        self.M = m[0] * m[1] * m[2]
        self.N = n[0] * n[1] * n[2]
        self.desc = ngf.level_desc(m, h, n, alpha, tau, rho)
        self.L = O.level(m, h, n, alpha, tau, rho)
        self.R = R.to(dev, torch.float32).contiguous()
        self.T = T.to(dev, torch.float32).contiguous()
        self.u = u.to(dev, torch.float32).contiguous()
        self.p = p.to(dev, torch.float32).contiguous()
        self.Rh, self.Th, self.uh, self.ph = f64(self.R), f64(self.T), f64(self.u), f64(self.p)

    def empty(self):
        return torch.empty(3 * self.N, device=self.R.device, dtype=torch.float32)


def random_case(m, h, n, alpha=0.7, tau=0.15, rho=0.25, seed=0, amp=0.3):
    g = torch.Generator().manual_seed(seed)
    M = m[0] * m[1] * m[2]
    N = n[0] * n[1] * n[2]
    R = torch.rand(M, generator=g)
    T = torch.rand(M, generator=g)
    u = amp * torch.randn(3 * N, generator=g) * min(h)
    p = torch.randn(3 * N, generator=g)
    return Case(m, h, n, alpha, tau, rho, R, T, u, p)


def workload_case(name, seed=5, amp_vox=0.5, dev="cuda"):
    """A named workload with a smooth random displacement of about amp_vox
    voxels (so warps are not identities) and a random direction p."""
    R, T, _, w = synth.make(name, device=dev)
    m, h, n = w["m"], w["h"], w["n"]
    N = n[0] * n[1] * n[2]
    u, p = synth.random_fields(N, seed, amp=amp_vox * min(h), device=dev)
    return Case(m, h, n, w["alpha"], w["tau"], w["rho"], R, T, u, p, dev=dev), w
