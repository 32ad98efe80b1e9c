"""Seeded synthetic inputs shared by the oracle tests, the CUDA path and the bench.

Holds random-number streams, scenes and camera paths only; none of the
rendering method's arithmetic lives here.
"""
from .rng import Stream, splitmix64, stream_seed
from .scenes import (FEAT_DIM, HIDDEN, IN_DIM, K_GAUSS, Model, city_scene,
                     glorot_mlps, head_out_dims, tiny_scene)
from .cameras import (Camera, HeadPose, city_path, look_rotation, path_extent,
                      pinhole, stereo_frames, stereo_pair, tiny_camera)


def city_workload(n_anchors: int = 2_000_000, seed: int = 10, path_seed: int = 11,
                  n_frames: int = 300, width: int = 1920, height: int = 1080):
    """The city-scale stereo workload: scene plus the ascending stereo path."""
    poses = city_path(n_frames=n_frames, seed=path_seed)
    x0, y0, x1, y1 = path_extent(poses)
    model = city_scene(n=n_anchors, seed=seed, keep_clear=(x0, y0, x1, y1, 30.0))
    frames = stereo_frames(poses, width=width, height=height)
    return model, frames


__all__ = [
    "Stream", "splitmix64", "stream_seed", "FEAT_DIM", "HIDDEN", "IN_DIM", "K_GAUSS",
    "Model", "city_scene", "glorot_mlps", "head_out_dims", "tiny_scene", "Camera",
    "HeadPose", "city_path", "look_rotation", "path_extent", "pinhole", "stereo_frames",
    "stereo_pair", "tiny_camera", "city_workload",
]
