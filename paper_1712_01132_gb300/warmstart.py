"""Learned warm start: a 3D convolutional U-Net that predicts the initial density and velocity
fields of the source iteration from the geometry and the Knudsen number.

The paper starts every run from h = 0 (Sec. 3.1) and spends many iterations near the continuum
limit, where the source iteration converges slowly.  Here a network trained on converged solutions
of the solver itself predicts (rho, u); dvm_set_initial turns the prediction into the state of an
iteration that produced the local equilibrium rho + 2 u.v.  The fixed point is unchanged, so the
converged answer does not depend on the network; only the iteration count does.

Network (all arithmetic in the library's CUDA kernels, torch only holds device memory):
  inputs   (solid mask, signed distance / 8, log10(Kn n1)), periodic grid
  outputs  (n1 (rho' - mean) / 4, 2 n1 u1, 2 n1 u2, 2 n1 u3) at the fluid voxels, where
           rho' = rho + x1 is the density in the solver's periodic source form (the pressure ramp
           removed).  The solver's length unit is the x1 period (n1 voxels), so per voxel the
           collision frequency is sqrt(pi) / (2 Kn n1) and the driving gradient 1 / n1: with
           Kn n1 as input and n1 rho', n1 u as outputs the network sees the same voxel-scale
           problem on any grid size and can be trained on smaller rocks than it is used on
  U-Net with `levels` levels and base * 2^l channels at level l, 3 x 3 x 3 periodic convolutions,
  ReLU, 2 x 2 x 2 mean pooling, nearest-neighbour upsampling, skip connections by concatenation;
  FP32 master weights, forward and backward on their BF16 roundings, FP32 accumulation; masked
  mean-squared error; Adam.
"""
import ctypes
import math

import numpy as np

from . import dvm

U_SCALE = 2.0       # velocity target = U_SCALE n1 u
R_SCALE = 0.25      # density target = R_SCALE n1 (rho' - mean)
SDF_SCALE = 8.0


def layer_shapes(levels, base, cin, cout):
    """(input channels, output channels) of every convolution, in parameter order: encoder levels
    0 .. L-1 (two convolutions each), decoder levels L-2 .. 0 (two each), output convolution."""
    ch = [base * 2 ** l for l in range(levels)]
    shapes = []
    for l in range(levels):
        shapes += [(cin if l == 0 else ch[l - 1], ch[l]), (ch[l], ch[l])]
    for l in reversed(range(levels - 1)):
        shapes += [(ch[l] + ch[l + 1], ch[l]), (ch[l], ch[l])]
    shapes.append((ch[0], cout))
    return shapes


def signed_distance(mask, cap=16):
    """Distance (voxels) to the nearest solid voxel in the fluid, minus the distance to the nearest
    fluid voxel in the solid, on the periodic grid, clipped to +-cap (a periodic margin of cap
    voxels around the grid makes every distance up to cap exact)."""
    from scipy import ndimage
    m = min(cap, *mask.shape)
    padded = np.pad(mask, m, mode="wrap")
    dfl = ndimage.distance_transform_edt(~padded)
    dso = ndimage.distance_transform_edt(padded)
    sl = tuple(slice(m, m + n) for n in mask.shape)
    return np.clip((dfl - dso)[sl], -cap, cap)


def features(mask, kn):
    """Network input [3][z][y][x] (float32)."""
    mask = np.asarray(mask, dtype=bool)
    return np.stack([mask.astype(np.float32), (signed_distance(mask) / SDF_SCALE).astype(np.float32),
                     np.full(mask.shape, math.log10(kn * mask.shape[-1]), np.float32)])


def targets(mask, kn, rho, u):
    """Training target [4][z][y][x] from converged moments in the paper's variables (rho carries
    the -x1 ramp; x1 = i / n1 on the cell index i)."""
    mask = np.asarray(mask, dtype=bool)
    fl = ~mask
    n1 = mask.shape[-1]
    x1 = np.broadcast_to(np.arange(n1) / n1, mask.shape)
    rp = (rho + x1) * fl
    rp = (rp - rp[fl].mean()) * fl
    return np.concatenate([R_SCALE * n1 * rp[None], U_SCALE * n1 * u * fl[None]]).astype(np.float32)


def to_initial(mask, kn, pred):
    """(rho0, u0) for dvm_set_initial from a network output [4][z][y][x]."""
    mask = np.asarray(mask, dtype=bool)
    fl = ~mask
    n1 = mask.shape[-1]
    x1 = np.broadcast_to(np.arange(n1) / n1, mask.shape)
    rho0 = (pred[0] / (R_SCALE * n1) - x1) * fl
    u0 = pred[1:] / (U_SCALE * n1) * fl[None]
    return rho0.astype(np.float64), u0.astype(np.float64)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class UNet:
    """The warm-start network on the GPU (one sample at a time)."""

    def __init__(self, levels=4, base=32, cin=3, cout=4, seed=0):
        import torch
        self.torch = torch
        self.lib = dvm.load()
        self.levels, self.base, self.cin, self.cout = levels, base, cin, cout
        self.shapes = layer_shapes(levels, base, cin, cout)
        rng = np.random.default_rng(seed)
        dev = torch.device("cuda")
        self.w, self.b = [], []
        for i, (ci, co) in enumerate(self.shapes):
            std = math.sqrt(2.0 / (ci * 27)) * (0.1 if i == len(self.shapes) - 1 else 1.0)
            self.w.append(torch.tensor(rng.standard_normal((co, ci, 27)) * std, dtype=torch.float32, device=dev))
            self.b.append(torch.zeros(co, dtype=torch.float32, device=dev))
        self.wq = [torch.empty_like(w) for w in self.w]
        self.dw = [torch.zeros_like(w) for w in self.w]
        self.db = [torch.zeros_like(b) for b in self.b]
        self.mw = [torch.zeros_like(w) for w in self.w]
        self.vw = [torch.zeros_like(w) for w in self.w]
        self.mb = [torch.zeros_like(b) for b in self.b]
        self.vb = [torch.zeros_like(b) for b in self.b]
        self.bq = [torch.empty_like(b) for b in self.b]
        self.steps = 0
        # per-channel standardisation of the targets (set from the training set): the network
        # learns (target - shift) / scale
        self.out_shift = np.zeros(cout, np.float32)
        self.out_scale = np.ones(cout, np.float32)
        self._requantize()

    # -- helpers
    @property
    def stream(self):
        return ctypes.c_void_p(self.torch.cuda.current_stream().cuda_stream)

    def _chk(self, st):
        if st != 0:
            raise dvm.DvmError(st, "network kernel failed")

    def _requantize(self):
        for w, q in zip(self.w + self.b, self.wq + self.bq):
            self._chk(self.lib.dvm_nn_round_bf16(_ptr(w), _ptr(q), w.numel(), self.stream))

    def _empty(self, c, dims):
        return self.torch.empty((c,) + tuple(dims), dtype=self.torch.float32, device="cuda")

    def _conv_scratch(self, ci, co, d, h, w):
        """The convolutions' scratch (padded BF16 input copy and BF16 weights), grown on demand."""
        n = int(self.lib.dvm_nn_conv3d_scratch_bytes(ci, co, d, h, w))
        if getattr(self, "_cscratch", None) is None or self._cscratch.numel() < n:
            self._cscratch = self.torch.empty(n, dtype=self.torch.uint8, device="cuda")
        return self._cscratch

    def _conv(self, x, p, y, relu):
        ci, co = self.shapes[p]
        d, h, w = x.shape[1:]
        sc = self._conv_scratch(ci, co, d, h, w)
        self._chk(self.lib.dvm_nn_conv3d(_ptr(x), _ptr(self.wq[p]), _ptr(self.bq[p]), _ptr(y), ci, co, d, h, w, 0,
                                         _ptr(sc), sc.numel(), self.stream))
        if relu:
            self._chk(self.lib.dvm_nn_relu(_ptr(y), y.numel(), self.stream))

    def parameters_for_reference(self):
        """[(w, b)] as float64 numpy arrays, the BF16-rounded values forward and backward use."""
        return [(q.double().cpu().numpy(), bq.double().cpu().numpy()) for q, bq in zip(self.wq, self.bq)]

    # -- forward / backward
    def forward(self, x):
        """x: device tensor [cin][d][h][w] (d, h, w divisible by 2^(levels-1)); returns [cout][d][h][w]."""
        L = self.levels
        ch = [self.base * 2 ** l for l in range(L)]
        self._rec = []
        dims = [tuple(x.shape[1:])]
        for l in range(1, L):
            dims.append(tuple(n // 2 for n in dims[-1]))
        # concatenation buffers of the decoder: [kept_l | up(h)]; the encoder writes kept_l in place
        self._cat = [self._empty(ch[l] + ch[l + 1], dims[l]) for l in range(L - 1)]
        h = x
        p = 0
        for l in range(L):
            a = self._empty(ch[l], dims[l])
            self._conv(h, p, a, True)
            self._rec.append((p, h, a))
            h, p = a, p + 1
            a = self._cat[l][:ch[l]] if l < L - 1 else self._empty(ch[l], dims[l])
            self._conv(h, p, a, True)
            self._rec.append((p, h, a))
            h, p = a, p + 1
            if l < L - 1:
                pooled = self._empty(ch[l], dims[l + 1])
                d, hh, w = dims[l]
                self._chk(self.lib.dvm_nn_pool2(_ptr(h), _ptr(pooled), ch[l], d, hh, w, self.stream))
                h = pooled
        for l in reversed(range(L - 1)):
            up = self._cat[l][ch[l]:]
            d, hh, w = dims[l]
            self._chk(self.lib.dvm_nn_up2(_ptr(h), _ptr(up), ch[l + 1], d, hh, w, self.stream))
            h = self._cat[l]
            for _ in range(2):
                a = self._empty(ch[l], dims[l])
                self._conv(h, p, a, True)
                self._rec.append((p, h, a))
                h, p = a, p + 1
        y = self._empty(self.cout, dims[0])
        self._conv(h, p, y, False)
        self._rec.append((p, h, None))
        self._dims = dims
        return y

    def _wgrad(self, p, x, g):
        ci, co = self.shapes[p]
        d, h, w = x.shape[1:]
        n = int(self.lib.dvm_nn_wgrad_scratch_floats(ci, co, d, h, w))
        if getattr(self, "_scratch", None) is None or self._scratch.numel() < n:
            self._scratch = self.torch.empty(n, dtype=self.torch.float32, device="cuda")
        self._chk(self.lib.dvm_nn_conv3d_wgrad(_ptr(x), _ptr(g), _ptr(self.dw[p]), _ptr(self.db[p]), _ptr(self._scratch),
                                               self._scratch.numel(), ci, co, d, h, w, 1, self.stream))

    def _dgrad(self, p, g, like):
        ci, co = self.shapes[p]
        d, h, w = g.shape[1:]
        dx = self._empty(ci, like)
        sc = self._conv_scratch(ci, co, d, h, w)
        self._chk(self.lib.dvm_nn_conv3d_dgrad(_ptr(g), _ptr(self.wq[p]), _ptr(dx), ci, co, d, h, w, 0, _ptr(sc),
                                               sc.numel(), self.stream))
        return dx

    def backward(self, dy):
        """Accumulates the parameter gradients of the last forward for the output gradient dy."""
        L = self.levels
        ch = [self.base * 2 ** l for l in range(L)]
        dims = self._dims
        rec = self._rec
        r = len(rec) - 1
        p, hin, _ = rec[r]
        self._wgrad(p, hin, dy)
        g = self._dgrad(p, dy, dims[0])
        r -= 1
        skip = {}
        for l in range(L - 1):                       # decoder levels 0 .. L-2, output side first
            for _ in range(2):
                p, hin, a = rec[r]
                self._chk(self.lib.dvm_nn_relu_bwd(_ptr(a), _ptr(g), g.numel(), self.stream))
                self._wgrad(p, hin, g)
                g = self._dgrad(p, g, hin.shape[1:])
                r -= 1
            skip[l] = g[:ch[l]]                       # gradient of kept_l
            gup = self._empty(ch[l + 1], dims[l + 1])
            d, hh, w = dims[l]
            self._chk(self.lib.dvm_nn_up2_bwd(_ptr(g[ch[l]:]), _ptr(gup), ch[l + 1], d, hh, w, self.stream))
            g = gup
        for l in reversed(range(L)):
            if l < L - 1:
                d, hh, w = dims[l]
                gk = skip[l].contiguous()
                self._chk(self.lib.dvm_nn_pool2_bwd(_ptr(g), _ptr(gk), ch[l], d, hh, w, 1, self.stream))
                g = gk
            for _ in range(2):
                p, hin, a = rec[r]
                self._chk(self.lib.dvm_nn_relu_bwd(_ptr(a), _ptr(g), g.numel(), self.stream))
                self._wgrad(p, hin, g)
                if r > 0:
                    g = self._dgrad(p, g, hin.shape[1:])
                r -= 1
        self._rec = None

    def zero_grad(self):
        for t in self.dw + self.db:
            t.zero_()

    def step(self, lr=1e-3, grad_scale=1.0, beta1=0.9, beta2=0.999, eps=1e-8):
        self.steps += 1
        for w, q, g, m, v in zip(self.w + self.b, self.wq + self.bq, self.dw + self.db, self.mw + self.mb,
                                 self.vw + self.vb):
            self._chk(self.lib.dvm_nn_adam(_ptr(w), _ptr(q), _ptr(g), _ptr(m), _ptr(v), w.numel(), lr, beta1, beta2,
                                           eps, self.steps, grad_scale, self.stream))

    def loss_and_grad(self, y, t, mask):
        """Masked mean-squared error of y against t over the fluid voxels and dL/dy."""
        torch = self.torch
        c = y.shape[0]
        V = y[0].numel()
        count = c * max(float(mask.sum().item()), 1.0)
        dy = torch.empty_like(y)
        nparts = int(self.lib.dvm_nn_mse_partials(c, V))
        part = torch.empty(nparts, dtype=torch.float32, device="cuda")
        self._chk(self.lib.dvm_nn_mse(_ptr(y), _ptr(t), _ptr(mask), _ptr(dy), _ptr(part), c, V, 1.0 / count,
                                      self.stream))
        return float(np.sum(part.cpu().numpy(), dtype=np.float64) / count), dy

    # -- persistence
    def set_standardisation(self, targets_and_masks):
        """Per-channel mean and standard deviation of the targets over the fluid voxels."""
        acc = np.zeros((self.cout, 3))
        for t, m in targets_and_masks:
            fl = m.reshape(t.shape[1:]) > 0
            for c in range(self.cout):
                x = t[c][fl].astype(np.float64)
                acc[c] += (x.size, x.sum(), (x * x).sum())
        mean = acc[:, 1] / acc[:, 0]
        self.out_shift = mean.astype(np.float32)
        self.out_scale = np.sqrt(np.maximum(acc[:, 2] / acc[:, 0] - mean ** 2, 1e-12)).astype(np.float32)

    def standardise(self, t):
        """Device target -> standardised device target."""
        sh = self.torch.tensor(self.out_shift, device="cuda")[:, None, None, None]
        sc = self.torch.tensor(self.out_scale, device="cuda")[:, None, None, None]
        return ((t - sh) / sc).contiguous()

    def destandardise(self, y):
        """Host network output -> target units."""
        return y * self.out_scale[:, None, None, None] + self.out_shift[:, None, None, None]

    def state(self):
        return {"levels": self.levels, "base": self.base, "cin": self.cin, "cout": self.cout,
                "out_shift": self.out_shift, "out_scale": self.out_scale,
                "w": [w.cpu().numpy() for w in self.w], "b": [b.cpu().numpy() for b in self.b]}

    def load_state(self, st):
        for w, a in zip(self.w, st["w"]):
            w.copy_(self.torch.from_numpy(np.asarray(a, dtype=np.float32)))
        for b, a in zip(self.b, st["b"]):
            b.copy_(self.torch.from_numpy(np.asarray(a, dtype=np.float32)))
        self._requantize()


def predict(net, mask, kn):
    """Network prediction [4][z][y][x] (numpy) for one geometry."""
    import torch
    x = torch.from_numpy(features(mask, kn)).cuda()
    y = net.forward(x)
    net._rec = None
    return net.destandardise(y.cpu().numpy())


def solve_to(mask, kn, v, w, tol, max_iter, initial=None, **options):
    """Run the solver to Err < tol (check interval 100); returns (iterations, seconds, k, rho, u)."""
    import time
    import torch
    s = dvm.Solver(mask, kn, v, w, **options)
    if initial is not None:
        s.set_initial(*initial)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, it, err = s.iterate(max_iter, tol)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    k = s.permeability()[0]
    rho, u = s.moments()
    s.close()
    return it, dt, k, rho, u, st


def training_set(train=48, side=64, nv=16, seed=0, kn_range=(0.05, 5.0), log=print):
    """Solver runs that make the training set: `train` seeded side^3 Gaussian-field rocks
    (correlation length 8, porosity 0.35, seeds 0, 1, ... without the non-percolating ones), Kn
    log-uniform in kn_range, nv^3 velocities, FP32, Err < 1e-6.  Returns (list of (features, target,
    fluid mask) device tensors, seconds)."""
    import time
    import torch
    from . import inputs
    v, w = dvm.dvm_gh_velocity_grid(3, nv)
    opts = dict(precision="fp32", lateral="periodic")
    rng = np.random.default_rng(seed)
    data = []
    t0 = time.perf_counter()
    rock_seed = 0
    while len(data) < train:
        # seeds whose field has no percolating pore space (all solid after the cluster filter) are
        # skipped
        mask = inputs.gaussian_rock(side, seed=rock_seed, corr_len=8.0, porosity=0.35)
        rock_seed += 1
        if mask.all():
            continue
        kn = float(10 ** rng.uniform(math.log10(kn_range[0]), math.log10(kn_range[1])))
        it, dt, k, rho, u, st = solve_to(mask, kn, v, w, 1e-6, 5000, **opts)
        data.append((torch.from_numpy(features(mask, kn)).cuda(), torch.from_numpy(targets(mask, kn, rho, u)).cuda(),
                     torch.from_numpy((~mask).astype(np.float32).ravel()).cuda()))
    t_data = time.perf_counter() - t0
    log("training set: %d runs in %.1f s" % (train, t_data))
    return data, t_data


def train_network(data, levels=4, base=16, steps=1500, lr=2e-3, constant_lr=False, seed=0, log=print):
    """Adam on the masked MSE of the standardised targets, one sample per step in turn.  Returns
    (network, dict with the step count, seconds and mean loss of the first and last epochs)."""
    import time
    import torch
    net = UNet(levels=levels, base=base, seed=seed)
    net.set_standardisation([(t.cpu().numpy(), m.cpu().numpy()) for _, t, m in data])
    data = [(x, net.standardise(t), m) for x, t, m in data]
    losses = []
    t0 = time.perf_counter()
    for step in range(steps):
        x, t, m = data[step % len(data)]
        net.zero_grad()
        y = net.forward(x)
        loss, dy = net.loss_and_grad(y, t, m)
        net.backward(dy)
        net.step(lr=lr if constant_lr else lr * 0.5 * (1.0 + math.cos(math.pi * step / steps)))
        losses.append(loss)
        if step % 200 == 0:
            log("step %d loss %.4e" % (step, loss))
    torch.cuda.synchronize()
    n = len(data)
    return net, {"levels": levels, "base": base, "steps": steps, "train_seconds": time.perf_counter() - t0,
                 "loss_first_epoch": float(np.mean(losses[:n])), "loss_last_epoch": float(np.mean(losses[-n:]))}


def time_to_tolerance(mask, kn, nv=16, net=None, tol=1e-6, ref_tol=1e-9, fp64=True, max_iter=20000,
                      fp32_options=None):
    """Iterations and wall time to Err < tol (Eq. 15, every 100 iterations) of the plain FP32 start,
    the plain FP64 start and (with a network) the warm FP32 start, on one geometry.  Wall time is
    the time of dvm_iterate (plus features, inference and dvm_set_initial for the warm start);
    context creation is reported separately.  The true permeability error of each stop
    (|k - k_ref| / k_ref, k_ref from the plain FP32 run continued to Err < ref_tol) shows whether
    Err < tol stopped near the fixed point."""
    import time
    import torch
    v, w = dvm.dvm_gh_velocity_grid(3, nv)
    o32 = dict(precision="fp32", lateral="periodic", use_graph=True)
    o32.update(fp32_options or {})
    out = {"tol": tol, "kn": kn, "fluid_cells": int((~np.asarray(mask, bool)).sum()), "velocities": len(w)}

    def run(opts, initial_fn=None, continue_to=None):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = dvm.Solver(mask, kn, v, w, **opts)
        torch.cuda.synchronize()
        setup = time.perf_counter() - t0
        t0 = time.perf_counter()
        extra = 0.0
        if initial_fn is not None:
            s.set_initial(*initial_fn())
            extra = time.perf_counter() - t0
        st, it, err = s.iterate(max_iter, tol)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        row = {"iterations": it, "seconds": dt, "setup_seconds": setup, "k": s.permeability()[0], "err": err,
               "converged": st == dvm.DVM_OK}
        if initial_fn is not None:
            row["features_inference_seconds"] = extra
        if continue_to is not None:
            st2, it2, err2 = s.iterate(max_iter, continue_to)
            row["k_ref"] = s.permeability()[0]
            row["k_ref_iterations"] = it + it2
            row["k_ref_err"] = err2
        s.close()
        return row

    plain = run(o32, continue_to=ref_tol)
    k_ref = plain.pop("k_ref")
    out["k_ref"] = {"k": k_ref, "iterations": plain.pop("k_ref_iterations"), "err": plain.pop("k_ref_err"),
                    "how": "plain FP32 run continued to Err < %g" % ref_tol}
    out["plain_fp32"] = plain
    if fp64:
        out["plain_fp64"] = run(dict(precision="fp64", lateral="periodic", use_graph=True))
    if net is not None:
        out["warm_fp32"] = run(o32, initial_fn=lambda: to_initial(mask, kn, predict(net, mask, kn)))
    for key in ("plain_fp32", "plain_fp64", "warm_fp32"):
        if key in out:
            out[key]["true_k_error"] = abs(out[key]["k"] - k_ref) / abs(k_ref)
    return out


def run_pipeline(train=48, side=64, eval_side=128, eval_seeds=(10000, 10001), eval_kns=(0.05, 0.5),
                 levels=4, base=16, steps=1500, lr=2e-3, nv=16, fp64=False, seed=0, log=print, constant_lr=False):
    """The learned-warm-start experiment: training set (training_set), network (train_network), then
    on held-out eval_side^3 rocks (seeds eval_seeds, Kn eval_kns) the plain and warm starts to
    Err < 1e-6 (time_to_tolerance, with the plain FP64 start when fp64 is set)."""
    from . import inputs
    data, t_data = training_set(train, side, nv, seed, log=log)
    net, info = train_network(data, levels, base, steps, lr, constant_lr, seed, log=log)
    res = dict(info, train_runs=train, train_side=side, data_seconds=t_data, eval=[])
    for sd in eval_seeds:
        mask = inputs.gaussian_rock(eval_side, seed=sd, corr_len=8.0, porosity=0.35)
        for kn in eval_kns:
            row = time_to_tolerance(mask, kn, nv, net=net, fp64=fp64)
            row["seed"] = sd
            fl = ~mask
            log(row)
            res["eval"].append(row)
    return res


def time_step(levels=3, base=24, side=64, steps=50, seed=0):
    """Time one training step (forward, masked loss, backward, Adam) and one forward pass of the
    network on a random side^3 input: returns milliseconds per step and per forward pass."""
    import time
    import torch
    net = UNet(levels=levels, base=base, seed=seed)
    rng = np.random.default_rng(seed)
    x = torch.tensor(rng.standard_normal((3, side, side, side)).astype(np.float32), device="cuda")
    t = torch.tensor(rng.standard_normal((4, side, side, side)).astype(np.float32), device="cuda")
    m = torch.tensor((rng.random(side ** 3) > 0.6).astype(np.float32), device="cuda")

    def step():
        net.zero_grad()
        y = net.forward(x)
        _, dy = net.loss_and_grad(y, t, m)
        net.backward(dy)
        net.step(lr=1e-4)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    torch.cuda.synchronize()
    ms_step = (time.perf_counter() - t0) / steps * 1e3
    t0 = time.perf_counter()
    for _ in range(steps):
        net.forward(x)
    torch.cuda.synchronize()
    ms_fwd = (time.perf_counter() - t0) / steps * 1e3
    return {"levels": levels, "base": base, "side": side, "ms_per_train_step": ms_step, "ms_per_forward": ms_fwd}


def time_convolutions(shapes=((32, 32, 64), (64, 64, 32), (128, 128, 16), (256, 256, 8), (96, 32, 64), (32, 64, 64)),
                      reps=20):
    """Time the library's convolution (dvm_nn_conv3d, its padded-copy and weight-copy kernels
    included) at the network's channel counts and grid sides (cin, cout, side): CUDA events around
    `reps` calls after three warm-ups.  Returns [{cin, cout, side, ms, tflops}]."""
    import torch
    lib = dvm.load()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = []
    for ci, co, n in shapes:
        x = torch.randn(ci, n, n, n, device="cuda")
        w = torch.randn(co, ci, 27, device="cuda") * 0.05
        b = torch.randn(co, device="cuda")
        y = torch.empty(co, n, n, n, device="cuda")
        nsc = lib.dvm_nn_conv3d_scratch_bytes(ci, co, n, n, n)
        sc = torch.empty(nsc, dtype=torch.uint8, device="cuda")
        args = [ctypes.c_void_p(t.data_ptr()) for t in (x, w, b, y)] + [ci, co, n, n, n, 0, ctypes.c_void_p(sc.data_ptr()),
                                                                        nsc, st]
        for _ in range(3):
            dvm._check(lib.dvm_nn_conv3d(*args), None)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            lib.dvm_nn_conv3d(*args)
        e1.record()
        torch.cuda.synchronize()
        if lib.dvm_nn_status(st) != 0:
            raise RuntimeError("convolution wait expired")
        ms = e0.elapsed_time(e1) / reps
        out.append({"cin": ci, "cout": co, "side": n, "ms": round(ms, 4),
                    "tflops": round(2.0 * n ** 3 * ci * co * 27 / ms / 1e9, 1)})
    return out


def main():
    import argparse
    import json
    ap = argparse.ArgumentParser(description="train and evaluate the learned warm start")
    ap.add_argument("--train", type=int, default=48)
    ap.add_argument("--side", type=int, default=64)
    ap.add_argument("--eval-side", type=int, default=128)
    ap.add_argument("--eval-seeds", type=int, nargs="+", default=[10000, 10001])
    ap.add_argument("--eval-kns", type=float, nargs="+", default=[0.05, 0.5])
    ap.add_argument("--levels", type=int, default=4)
    ap.add_argument("--base", type=int, default=16)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--nv", type=int, default=16)
    ap.add_argument("--fp64", action="store_true", help="also time the plain FP64 start to tolerance")
    ap.add_argument("--constant-lr", action="store_true")
    ap.add_argument("--out", default=None)
    ap.add_argument("--time-step", action="store_true",
                    help="only time a training step and a forward pass of the network (--levels, --base, --side)")
    ap.add_argument("--time-conv", action="store_true",
                    help="only time the convolution entry point at the network's channel counts")
    a = ap.parse_args()
    if a.time_conv:
        for row in time_convolutions():
            print(json.dumps(row))
        return
    if a.time_step:
        import json
        print(json.dumps(time_step(a.levels, a.base, a.side)))
        return
    res = run_pipeline(a.train, a.side, a.eval_side, tuple(a.eval_seeds), tuple(a.eval_kns), a.levels, a.base,
                       a.steps, a.lr, a.nv, a.fp64, constant_lr=a.constant_lr)
    text = json.dumps(res, indent=1)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text)
    print(text)


if __name__ == "__main__":
    main()
