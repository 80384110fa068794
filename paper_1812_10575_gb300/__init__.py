"""GB300-native Random Batch Method (RBM-1) hot path (arXiv:1812.10575).

The compute lives in ``librbm.so`` (hand-written sm_103a CUDA behind the C ABI
of ``include/rbm.h``); this package is its thin Python binding plus a small
convenience wrapper, :class:`System`.  PyTorch supplies device memory and
streams only.

    import torch, paper_1812_10575_gb300 as rbm
    x = torch.randn(4096, 4, device="cuda")            # N x ld, d = 3
    sysm = rbm.System(x, d=3, p=2, dt=1e-3, k="coulomb", renorm=True)
    sysm.run(100)                                        # 100 RBM-1 steps
    sysm.sync()
"""
from __future__ import annotations

from ._lib import (  # noqa: F401
    EXPORTS, KERNELS, METHODS, POTENTIALS, SCHEMES, RbmError, RbmParams, RbmTuning, library_path, load,
    make_params, rbm_direct_forces_at, rbm_direct_step, rbm_forces, rbm_free, rbm_get_step, rbm_get_tuning,
    rbm_init, rbm_last_error, rbm_launches_per_step, rbm_permutation, rbm_permutation_noalloc, rbm_run, rbm_set_step, rbm_set_tuning,
    rbm_status_string, rbm_step, rbm_step_host, rbm_step_profiled, rbm_sync, rbm_batched_init,
    rbm_batched_set_launch, rbm_autotune, rbm_surrogate_config, rbm_surrogate_train, rbm_surrogate_stats,
    rbm_surrogate_params, rbm_surrogate_set_params, rbm_surrogate_forces, rbm_surrogate_gradient,
    rbm_rbmr_sets, rbm_rbmr_info, rbm_verlet_set_velocity, rbm_verlet_get_previous, rbm_verlet_set_previous,
    rbm_surrogate_save, rbm_surrogate_load, rbm_latency_floor, rbm_set_noise_refinement, rbm_get_noise_refinement,
    rbm_surrogate_drift, rbm_set_batch_size, rbm_autotune_accuracy, rbm_fp32_fma_peak,
    N_SURROGATE_PARAMS,
)


def leading_dim(d: int) -> int:
    """Row length of the position array: d for d = 1, 2 and 4 for d = 3."""
    return 4 if d == 3 else d


class Replicas:
    """Independent systems of sizes ``sizes`` in one caller-owned CUDA tensor
    ``x`` of shape ``(sum(sizes), leading_dim(d))``, advanced together."""

    def __init__(self, x, sizes, d, p=2, dt=1e-3, sigma=0.0, seed=0, v="zero", v_coef=1.0, k="linear",
                 k_param=0.0, renorm=False, stream=None):
        import torch

        self.x = x
        self.d = d
        self.sizes = [int(v) for v in sizes]
        if x.dim() != 2 or x.shape[0] != sum(self.sizes) or x.shape[1] != leading_dim(d):
            raise ValueError("positions must have shape (sum(sizes), leading_dim(d))")
        self.params = make_params(sum(self.sizes), d, p=p, dt=dt, sigma=sigma, seed=seed,
                                  dtype="f32" if x.dtype == torch.float32 else "f64", v=v, v_coef=v_coef, k=k,
                                  k_param=k_param, renorm=renorm)
        self.ctx = rbm_batched_init(self.params, self.sizes, x, stream)

    def step(self):
        rbm_step(self.ctx)

    def run(self, steps):
        rbm_run(self.ctx, steps, "rbm")

    def sync(self):
        rbm_sync(self.ctx)

    @property
    def m(self):
        return rbm_get_step(self.ctx)

    @m.setter
    def m(self, value):
        rbm_set_step(self.ctx, value)

    def permutation(self):
        import torch

        perm = torch.empty(self.x.shape[0], dtype=torch.int32, device=self.x.device)
        rbm_permutation(self.ctx, perm)
        return perm

    def forces(self):
        import torch

        f = torch.zeros_like(self.x)
        rbm_forces(self.ctx, "rbm", f)
        return f

    def set_launch(self, threads, bucket_target):
        rbm_batched_set_launch(self.ctx, threads, bucket_target)

    def set_noise_refinement(self, r):
        rbm_set_noise_refinement(self.ctx, r)

    def set_batch_size(self, p):
        rbm_set_batch_size(self.ctx, p)

    def autotune_accuracy(self, ps, eps, horizon, **kw):
        return rbm_autotune_accuracy(self.ctx, ps, eps, horizon, **kw)

    def set_graph_steps(self, steps):
        rbm_set_tuning(self.ctx, RbmTuning(graph_steps=steps))

    def autotune(self, trial_steps=3, table_path=None):
        return rbm_autotune(self.ctx, trial_steps, table_path)


    def step_profiled(self):
        return rbm_step_profiled(self.ctx, "rbm")

    def close(self):
        if getattr(self, "ctx", None) is not None:
            rbm_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class System:
    """One particle system bound to a caller-owned CUDA tensor ``x`` of shape
    ``(N, leading_dim(d))``.  Methods map one-to-one onto the C entry points."""

    def __init__(self, x, d, p=2, dt=1e-3, sigma=0.0, seed=0, v="zero", v_coef=1.0, k="linear",
                 k_param=0.0, renorm=False, scheme="euler", replica=0, gbm=False, stream=None):
        import torch

        if x.dtype not in (torch.float32, torch.float64):
            raise ValueError("positions must be float32 or float64")
        if x.dim() != 2 or x.shape[1] != leading_dim(d):
            raise ValueError(f"positions must have shape (N, {leading_dim(d)})")
        self.x = x
        self.d = d
        self.params = make_params(x.shape[0], d, p=p, dt=dt, sigma=sigma, seed=seed,
                                  dtype="f32" if x.dtype == torch.float32 else "f64", v=v, v_coef=v_coef,
                                  k=k, k_param=k_param, renorm=renorm, scheme=scheme, replica=replica, gbm=gbm)
        self.ctx = rbm_init(self.params, x, stream)

    def step(self):
        rbm_step(self.ctx)

    def direct_step(self):
        rbm_direct_step(self.ctx)

    def run(self, steps, method="rbm"):
        rbm_run(self.ctx, steps, method)

    def step_host(self, x_host, method="rbm"):
        rbm_step_host(self.ctx, x_host, method)

    @property
    def m(self):
        return rbm_get_step(self.ctx)

    @m.setter
    def m(self, value):
        rbm_set_step(self.ctx, value)

    def sync(self):
        rbm_sync(self.ctx)

    def permutation(self):
        import torch

        perm = torch.empty(self.x.shape[0], dtype=torch.int32, device=self.x.device)
        rbm_permutation(self.ctx, perm)
        return perm

    def forces(self, method="rbm"):
        import torch

        f = torch.zeros_like(self.x)
        rbm_forces(self.ctx, method, f)
        return f

    def direct_forces_at(self, q):
        import torch

        f = torch.zeros_like(q)
        rbm_direct_forces_at(self.ctx, q, f)
        return f

    def set_tuning(self, **kw):
        t = RbmTuning(**kw)
        rbm_set_tuning(self.ctx, t)

    def set_noise_refinement(self, r):
        """Brownian increments shared with a run of step dt/r (path coupling)."""
        rbm_set_noise_refinement(self.ctx, r)

    def set_batch_size(self, p):
        rbm_set_batch_size(self.ctx, p)

    def autotune_accuracy(self, ps, eps, horizon, **kw):
        return rbm_autotune_accuracy(self.ctx, ps, eps, horizon, **kw)

    def tuning(self):
        t = rbm_get_tuning(self.ctx)
        return {f: getattr(t, f) for f, _ in RbmTuning._fields_}

    def step_profiled(self, method="rbm"):
        return rbm_step_profiled(self.ctx, method)

    def autotune(self, trial_steps=3, table_path=None):
        return rbm_autotune(self.ctx, trial_steps, table_path)

    def launches_per_step(self, method="rbm"):
        return rbm_launches_per_step(self.ctx, method)

    # second-order system, scheme="verlet": velocities before the first step
    def verlet_set_velocity(self, v):
        if v.shape != self.x.shape or v.dtype != self.x.dtype or not v.is_contiguous():
            raise ValueError("velocities must match the positions' shape, dtype and layout")
        rbm_verlet_set_velocity(self.ctx, v)

    def verlet_get_previous(self):
        """(X_{n-1} or V_0, Taylor start pending) for checkpoint/resume."""
        import torch

        prev = torch.empty_like(self.x)
        pending = rbm_verlet_get_previous(self.ctx, prev)
        return prev, pending

    def verlet_set_previous(self, prev, taylor_pending):
        rbm_verlet_set_previous(self.ctx, prev.contiguous(), taylor_pending)

    def latency_floor(self):
        return rbm_latency_floor(self.ctx)

    def surrogate_save(self):
        return rbm_surrogate_save(self.ctx)

    def surrogate_load(self, state):
        rbm_surrogate_load(self.ctx, state)

    # RBM-r (Algorithm "fullyrandom"): run(steps, "rbmr")
    def rbmr_info(self):
        return rbm_rbmr_info(self.ctx)

    def rbmr_sets(self, m):
        import torch

        k = rbm_rbmr_info(self.ctx)["iterations_per_step"]
        sets = torch.empty(k, self.params.p, dtype=torch.int32, device=self.x.device)
        rbm_rbmr_sets(self.ctx, m, sets)
        return sets

    # learned mean-field surrogate (d = 2 or 3, FP32)
    def surrogate_config(self, **kw):
        rbm_surrogate_config(self.ctx, **kw)

    def surrogate_train(self, iters):
        rbm_surrogate_train(self.ctx, iters)

    def surrogate_stats(self):
        return rbm_surrogate_stats(self.ctx)

    def surrogate_drift(self):
        return rbm_surrogate_drift(self.ctx)

    def surrogate_params(self):
        return rbm_surrogate_params(self.ctx, self.d)

    def surrogate_set_params(self, theta, norm=None):
        rbm_surrogate_set_params(self.ctx, theta, norm, self.d)

    def surrogate_forces(self, q):
        import torch

        f = torch.zeros_like(q)
        rbm_surrogate_forces(self.ctx, q, f)
        return f

    def surrogate_gradient(self, x, f_target):
        return rbm_surrogate_gradient(self.ctx, x, f_target, self.d)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            rbm_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
