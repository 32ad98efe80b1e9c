"""Seeded camera rigs and camera paths (inputs, not method arithmetic).

Convention: world z is up; a camera maps world x to camera coordinates
c = R x + t with camera x right, y down, z forward; the pixel centre of
pixel (i, j) is at (i + 0.5, j + 0.5).  Every value handed to the renderer is
float32; poses are built in float64 and cast once.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List

import numpy as np

from .rng import Stream


@dataclass
class Camera:
    R: np.ndarray        # float32 [3,3] world -> camera rotation (rows: right, down, forward)
    t: np.ndarray        # float32 [3]
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    znear: float = 0.2

    @property
    def center(self) -> np.ndarray:
        R = self.R.astype(np.float64)
        return -R.T @ self.t.astype(np.float64)


def _f32(x) -> float:
    return float(np.float32(x))


def look_rotation(yaw: float, pitch: float) -> np.ndarray:
    """Rows (right, down, forward) for heading `yaw` (rad from +x) and `pitch` (rad, <0 looks down)."""
    f = np.array([np.cos(pitch) * np.cos(yaw), np.cos(pitch) * np.sin(yaw), np.sin(pitch)])
    r = np.array([np.sin(yaw), -np.cos(yaw), 0.0])
    d = np.cross(f, r)
    return np.stack([r, d, f], axis=0)


def pinhole(R64: np.ndarray, center: np.ndarray, width: int, height: int, hfov_deg: float,
            znear: float = 0.2) -> Camera:
    fx = (width / 2.0) / np.tan(np.deg2rad(hfov_deg) / 2.0)
    R32 = R64.astype(np.float32)
    t = -(R32.astype(np.float64) @ np.asarray(center, np.float64))
    return Camera(R=R32, t=t.astype(np.float32), fx=_f32(fx), fy=_f32(fx),
                  cx=_f32(width / 2.0), cy=_f32(height / 2.0), width=int(width),
                  height=int(height), znear=_f32(znear))


def tiny_camera(width: int = 256, height: int = 256, hfov_deg: float = 60.0) -> Camera:
    """One pinhole at (0, 0, -15) looking along +z (world axes as camera axes)."""
    R = np.eye(3)
    return pinhole(R, np.array([0.0, 0.0, -15.0]), width, height, hfov_deg)


def stereo_pair(R64: np.ndarray, head: np.ndarray, width: int, height: int,
                hfov_deg: float, baseline: float = 0.064):
    """Left/right eyes sharing R, separated by `baseline` along camera right."""
    right = R64[0]
    left = pinhole(R64, head - right * baseline / 2.0, width, height, hfov_deg)
    rght = pinhole(R64, head + right * baseline / 2.0, width, height, hfov_deg)
    return left, rght


@dataclass
class HeadPose:
    pos: np.ndarray     # float64 [3]
    yaw: float
    pitch: float


def city_path(n_frames: int = 300, seed: int = 11, start=(-600.0, -600.0),
              h0: float = 2.0, h1: float = 300.0, speed: float = 0.25,
              yaw0_deg: float = 45.0, yaw_rate_deg: float = 0.15,
              pitch0_deg: float = -5.0, pitch1_deg: float = -35.0) -> List[HeadPose]:
    """Ascending aerial path: altitude h_t = h0 (h1/h0)^(t/(n-1)), horizontal
    speed `speed` m/frame, yaw and pitch changing linearly (<= 0.5 deg/frame
    combined).  A small seeded wobble (<= 0.05 deg) keeps frames distinct."""
    st = Stream(seed, "path")
    wob = st.normal(2 * n_frames, 0.0, 0.02).reshape(n_frames, 2)
    poses = []
    x, y = start
    yaw = np.deg2rad(yaw0_deg)
    for t in range(n_frames):
        s = t / max(n_frames - 1, 1)
        h = h0 * (h1 / h0) ** s
        pitch = np.deg2rad(pitch0_deg + (pitch1_deg - pitch0_deg) * s + wob[t, 0])
        yw = yaw + np.deg2rad(wob[t, 1])
        poses.append(HeadPose(pos=np.array([x, y, h]), yaw=float(yw), pitch=float(pitch)))
        x += speed * np.cos(yaw)
        y += speed * np.sin(yaw)
        yaw += np.deg2rad(yaw_rate_deg)
    return poses


def path_extent(poses: List[HeadPose]):
    p0, p1 = poses[0].pos, poses[-1].pos
    return float(p0[0]), float(p0[1]), float(p1[0]), float(p1[1])


def stereo_frames(poses: List[HeadPose], width: int = 1920, height: int = 1080,
                  hfov_deg: float = 60.0, baseline: float = 0.064):
    """List of (left, right) Camera pairs along a path."""
    return [stereo_pair(look_rotation(p.yaw, p.pitch), p.pos, width, height, hfov_deg, baseline)
            for p in poses]


def reuse_path(seed: int = 12, n_frames: int = 120, speed: float = 1.0) -> List[HeadPose]:
    """Ascending city path (same corridor as `city_path(seed=11)`) with a
    seeded look-around: the head yaw swings A sin(2 pi t / P + phi) about the
    heading (A 45-60 deg, P 24-32 frames), the pitch B sin(2 pi t / Q + psi)
    (B 4-8 deg), so consecutive frames share roughly 80-95% of their visible
    anchors.  Seed 12: the evaluation path of the cached form; seeds 20-29:
    training paths of the reuse predictor; seed 30: its held-out path."""
    st = Stream(seed, "look")
    A, P, phi = np.deg2rad(st.uniform(1, 45.0, 60.0)[0]), st.uniform(1, 24.0, 32.0)[0], st.uniform(1, 0.0, 2 * np.pi)[0]
    B, Q, psi = np.deg2rad(st.uniform(1, 4.0, 8.0)[0]), st.uniform(1, 30.0, 50.0)[0], st.uniform(1, 0.0, 2 * np.pi)[0]
    start = st.uniform(1, 0.0, 150.0)[0]  # metres along the corridor
    base = city_path(n_frames=n_frames, seed=11, speed=speed)
    d = np.array([np.cos(np.deg2rad(45.0)), np.sin(np.deg2rad(45.0)), 0.0])
    out = []
    for t, q in enumerate(base):
        out.append(HeadPose(pos=q.pos + start * d, yaw=q.yaw + A * np.sin(2 * np.pi * t / P + phi),
                            pitch=q.pitch + B * np.sin(2 * np.pi * t / Q + psi)))
    return out
