"""The five workload presets (plain data; no arithmetic of the method).

cfg1  plain FP32 forward: L8 F2 T2^14 Nmin16 b1.5, MLP 16-64-64-1, params U(+-0.1),
      2^16 uniform points, 64x64 orthographic march of 128 steps, ramp LUT
cfg2  training: 128^3 blob volume, L16 F2 T2^19 Nmin16 b1.38, MLP 32-64-64-1,
      2^18 points per step, L2 loss, Adam lr 1e-2, FP32 and FP16 MLP
cfg3  mixed-precision render: 512^3 blob volume, cfg2's encoding at T2^21,
      FP16 / BF16 MLP, 1920x1080 perspective, step 0.5 voxel, 16^3 macrocells,
      early termination at 0.99
cfg4  in-loop training: 1024^3 blob volume, L16 F4 T2^22, MLP 64-64-64-1 FP16;
      per frame one 2^18-point step + a 1024x1024 render
cfg5  out-of-core training: 2048^3 blob volume in host memory as 64^3 bricks,
      L16 F4 T2^23, MLP 64-64-64-1 BF16, 2^19 points per step
"""
from dataclasses import dataclass, field


@dataclass(frozen=True)
class NetCfg:
    L: int
    F: int
    log2T: int
    Nmin: int
    b: float
    dims: tuple

    def kwargs(self):
        return dict(L=self.L, F=self.F, log2T=self.log2T, Nmin=self.Nmin, b=self.b, dims=self.dims)


CFG1_NET = NetCfg(8, 2, 14, 16, 1.5, (16, 64, 64, 1))
CFG2_NET = NetCfg(16, 2, 19, 16, 1.38, (32, 64, 64, 1))
CFG3_NET = NetCfg(16, 2, 21, 16, 1.38, (32, 64, 64, 1))
CFG4_NET = NetCfg(16, 4, 22, 16, 1.38, (64, 64, 64, 1))
CFG5_NET = NetCfg(16, 4, 23, 16, 1.38, (64, 64, 64, 1))

CFG1 = dict(net=CFG1_NET, n_points=1 << 16, param_seed=1, point_seed=2, image=(64, 64), steps=128)
CFG2 = dict(net=CFG2_NET, volume=128, volume_seed=3, batch=1 << 18, lr=1e-2, steps=1000)
CFG3 = dict(net=CFG3_NET, volume=512, volume_seed=4, image=(1920, 1080), vfov=40.0,
            eye=(0.5, 0.5, -1.0), target=(0.5, 0.5, 0.5), step_voxels=0.5, cell=16, et=0.99, K=8,
            alpha_floor=0.1, train_steps=2000, batch=1 << 18)
CFG4 = dict(net=CFG4_NET, volume=1024, volume_seed=5, image=(1024, 1024), batch=1 << 18, frames=500,
            step_voxels=0.5, cell=16, et=0.99, K=8, alpha_floor=0.1)
CFG5 = dict(net=CFG5_NET, volume=2048, volume_seed=6, brick=64, ring=4096, refresh=256, batch=1 << 19)
