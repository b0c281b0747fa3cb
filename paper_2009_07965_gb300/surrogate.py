"""Learned basis surrogate: a 4-layer, 32-channel convolutional network that
maps a full interior leaf's permeability patch (with a one-cell halo) and
alpha to its 16 basis response fields, trained on fields the plain method
computes, with a residual gate in front of the plain local solve.

Every arithmetic step runs in libmrcm's kernels (BF16 tensor-core
convolutions, their gradients, Adam); this module holds the parameters and
activations (torch tensors used as device memory) and calls them in order.

Network: conv3x3 16->32 'valid' (the 18 x 18 input with its halo gives the
16 x 16 leaf) + ReLU, two conv3x3 32->32 'same' + ReLU, conv3x3 32->16
'same' (linear): output [item][16][16][16] = the fields psi_s at every cell
(layout of mrcm_leaf_fields).
"""
import numpy as np
import torch

from . import binding as B

LAYERS = [(16, 32, 0, True), (32, 32, 1, True), (32, 32, 1, True), (32, 16, 1, False)]   # cin, cout, pad, relu


class BasisSurrogate:
    def __init__(self, device="cuda", seed=0):
        dev = torch.device(device)
        self.device = dev
        rng = np.random.default_rng(seed)
        self.w, self.b, self.wbf, self.flip = [], [], [], []
        self.mw, self.vw, self.mb, self.vb = [], [], [], []
        for cin, cout, pad, relu in LAYERS:
            fan_in = 9 * cin
            w = rng.standard_normal((cout, 3, 3, cin)).astype(np.float32) * np.float32(np.sqrt(2.0 / fan_in))
            if cin == 16 and pad == 0:
                w[:, :, :, 2:] = 0.0            # input channels beyond the two used carry nothing
            wt = torch.from_numpy(w).to(dev).contiguous()
            self.w.append(wt)
            self.b.append(torch.zeros(cout, dtype=torch.float32, device=dev))
            self.wbf.append(wt.to(torch.bfloat16))
            self.flip.append(torch.empty((cin, 3, 3, cout), dtype=torch.bfloat16, device=dev))
            self.mw.append(torch.zeros_like(wt))
            self.vw.append(torch.zeros_like(wt))
            self.mb.append(torch.zeros(cout, dtype=torch.float32, device=dev))
            self.vb.append(torch.zeros(cout, dtype=torch.float32, device=dev))
        self.step = 0

    def _stream(self):
        return torch.cuda.current_stream(self.device).cuda_stream

    def forward(self, x, keep=False):
        """x: bf16 [count][18][18][16] patches -> float [count][16][16][16]."""
        count = x.shape[0]
        acts = [x]
        s = self._stream()
        for li, (cin, cout, pad, relu) in enumerate(LAYERS):
            last = li == len(LAYERS) - 1
            if last:
                y = torch.empty((count, 16, 16, cout), dtype=torch.float32, device=self.device)
                B.mrcm_cnn_conv_forward(acts[-1], count, cin, cout, pad, relu, self.wbf[li], self.b[li], None, y, s)
            else:
                y = torch.empty((count, 16, 16, cout), dtype=torch.bfloat16, device=self.device)
                B.mrcm_cnn_conv_forward(acts[-1], count, cin, cout, pad, relu, self.wbf[li], self.b[li], y, None, s)
            acts.append(y)
        return (acts[-1], acts) if keep else acts[-1]

    def train_step(self, x, target, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        """One Adam step on the mean squared error of the fields; returns the
        loss (a host float, read after the step)."""
        count = x.shape[0]
        s = self._stream()
        pred, acts = self.forward(x, keep=True)
        loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        dpost = torch.empty_like(pred)
        B.mrcm_cnn_mse_grad(pred, target, count, dpost, loss, s)
        dws = [torch.zeros_like(w) for w in self.w]
        dbs = [torch.zeros_like(b) for b in self.b]
        for li in range(len(LAYERS) - 1, -1, -1):
            cin, cout, pad, relu = LAYERS[li]
            dpre = torch.empty(dpost.shape, dtype=torch.bfloat16, device=self.device)
            # the layer's output acts[li + 1]: its ReLU mask (none on the last)
            B.mrcm_cnn_relu_grad(dpost, acts[li + 1], dpost.numel(), relu, dpre, s)
            B.mrcm_cnn_conv_wgrad(acts[li], dpre, count, cin, cout, pad, dws[li], dbs[li], s)
            if li > 0:
                B.mrcm_cnn_flip_weights(self.wbf[li], cout, cin, self.flip[li], s)
                dpost = torch.empty((count, 16, 16, cin), dtype=torch.float32, device=self.device)
                B.mrcm_cnn_conv_forward(dpre, count, cout, cin, 1, False, self.flip[li], None, None, dpost, s)
        self.step += 1
        for li in range(len(LAYERS)):
            B.mrcm_cnn_adam(self.w[li], dws[li], self.mw[li], self.vw[li], self.wbf[li], self.w[li].numel(), lr,
                            beta1, beta2, eps, self.step, s)
            B.mrcm_cnn_adam(self.b[li], dbs[li], self.mb[li], self.vb[li], None, self.b[li].numel(), lr, beta1,
                            beta2, eps, self.step, s)
        return float(loss.item())

    def predict(self, ctx, leaf_ids):
        """Fields of the given interior leaves (device int tensor of ids)."""
        x = torch.empty((leaf_ids.numel(), 18, 18, 16), dtype=torch.bfloat16, device=self.device)
        B.mrcm_leaf_patches(ctx, leaf_ids, x)
        return self.forward(x)

    def apply(self, ctx, leaf_ids, tau):
        """Predicts the fields of the leaves, gates them at relative residual
        tau and puts the accepted leaves' maps into the context (the merges
        are rebuilt; the others keep the plain local solve's maps).  Returns
        (accepted mask, residuals) as host arrays."""
        psi = self.predict(ctx, leaf_ids)
        res = torch.empty(leaf_ids.numel(), dtype=torch.float64, device=self.device)
        B.mrcm_leaf_gate(ctx, leaf_ids, psi, res)
        acc = torch.empty(leaf_ids.numel(), dtype=torch.int32, device=self.device)
        B.mrcm_leaf_apply(ctx, leaf_ids, psi, res, tau, acc)
        return acc.cpu().numpy().astype(bool), res.cpu().numpy()
