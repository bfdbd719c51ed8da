"""Seeded synthetic densities for the periodic L2 optimal-transport solver.

This module holds input generation only: a counter-based random generator and the
closed-form or image-like test densities.  It contains none of the solver's arithmetic and
is shared, as data, by the CPU oracle's tests and the GPU path's tests and benchmark.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15, then two xor-shift-multiply
rounds; a double in [0, 1) is the top 53 bits times 2^-53.

Grid convention: arrays are (N, M) float64; row index i is y = i/N, column index j is
x = j/M.

Workloads (the paper's own images -- BrainWeb MRI slices and two photographs -- are not
available, so these stand in for them, with image-like shapes and a positive floor):
  manufactured(N, M)       closed-form solution of the manufactured example (Sec. 5.1)
  blob_pair(N, M, s)       mixtures of 8 periodic Gaussian blobs plus a floor of 0.1
  noise_blob_pair(N, M, s) Gaussian-smoothed uniform noise plus 16 blobs, max/min = 10
"""
import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """Counter-based SplitMix64 stream."""

    def __init__(self, seed):
        self.state = int(seed) & _MASK

    def next_u64(self, n):
        """n consecutive outputs as a uint64 numpy array (vectorised over the counter)."""
        gamma = np.uint64(0x9E3779B97F4A7C15)
        k = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = np.uint64(self.state) + k * gamma
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        self.state = (self.state + n * 0x9E3779B97F4A7C15) & _MASK
        return z

    def uniform(self, n):
        return (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def grid(N, M):
    """(x, y) coordinate arrays of the N x M periodic grid."""
    y, x = np.meshgrid(np.arange(N) / N, np.arange(M) / M, indexing="ij")
    return x, y


# ----------------------------------------------------------------------------------------
# Manufactured example (Sec. 5.1 with explicit constants)
# ----------------------------------------------------------------------------------------
MANUFACTURED_A = 0.02 / (2.0 * np.pi) ** 2


def manufactured(N, M, amp=MANUFACTURED_A, g_amp=0.5):
    """phi*(x,y) = amp sin(2 pi x) sin(2 pi y); g = 1 + g_amp cos(2 pi x) cos(2 pi y);
    f = g(x + grad phi*) det(I + D^2 phi*) evaluated analytically (the problem's definition
    applied to the chosen phi*, so that phi* is the exact solution of the continuous
    problem).  Returns (f, g, phi*)."""
    x, y = grid(N, M)
    tp = 2.0 * np.pi
    phi = amp * np.sin(tp * x) * np.sin(tp * y)
    px = tp * amp * np.cos(tp * x) * np.sin(tp * y)
    py = tp * amp * np.sin(tp * x) * np.cos(tp * y)
    pxx = -tp * tp * amp * np.sin(tp * x) * np.sin(tp * y)
    pyy = pxx
    pxy = tp * tp * amp * np.cos(tp * x) * np.cos(tp * y)

    def gfun(a, b):
        return 1.0 + g_amp * np.cos(tp * a) * np.cos(tp * b)

    det = (1.0 + pxx) * (1.0 + pyy) - pxy * pxy
    f = gfun(x + px, y + py) * det
    g = gfun(x, y)
    return f, g, phi


# ----------------------------------------------------------------------------------------
# Blob mixtures
# ----------------------------------------------------------------------------------------
def periodic_gaussian(N, M, cx, cy, sigma, images=2):
    """exp(-|x - c + p|^2 / (2 sigma^2)) summed over the integer shifts p in
    {-images..images}^2 (truncation below e^-70 for sigma <= 0.12), evaluated as the
    product of the two 1-D periodic sums (the 2-D sum factorises)."""
    x = np.arange(M) / M
    y = np.arange(N) / N
    gx = np.zeros(M)
    gy = np.zeros(N)
    for p in range(-images, images + 1):
        gx += np.exp(-((x - cx + p) ** 2) / (2.0 * sigma * sigma))
        gy += np.exp(-((y - cy + p) ** 2) / (2.0 * sigma * sigma))
    return gy[:, None] * gx[None, :]


def blobs(N, M, rng, count, weight_scale=1.0):
    """sum of `count` periodic Gaussians; per blob the draws are, in order, centre x,
    centre y (uniform on the torus), sigma ~ U[0.03, 0.12], weight ~ U[0.5, 2]."""
    out = np.zeros((N, M))
    for _ in range(count):
        cx, cy, s, w = rng.uniform(4)
        sigma = 0.03 + 0.09 * s
        weight = (0.5 + 1.5 * w) * weight_scale
        out += weight * periodic_gaussian(N, M, cx, cy, sigma)
    return out


def blob_density(N, M, seed, count=8, floor=0.1):
    d = floor + blobs(N, M, SplitMix64(seed), count)
    return d / d.mean()


def blob_pair(N, M, s=1000):
    """Image-pair workload: f from seed 2s, g from seed 2s+1, each 0.1 + 8 blobs, mean 1."""
    return blob_density(N, M, 2 * s), blob_density(N, M, 2 * s + 1)


# ----------------------------------------------------------------------------------------
# Smoothed noise + blobs
# ----------------------------------------------------------------------------------------
def smoothed_noise(N, M, rng, sigma_px=8.0):
    """Uniform noise U[0,1) (row-major draws) convolved periodically with a Gaussian of
    standard deviation sigma_px pixels (multiplier exp(-2 pi^2 sigma^2 (k1^2/M^2 +
    k2^2/N^2)) on the discrete spectrum), then rescaled to [0, 1]."""
    z = rng.uniform(N * M).reshape(N, M)
    k1 = np.fft.fftfreq(M)  # cycles per pixel
    k2 = np.fft.fftfreq(N)
    mult = np.exp(-2.0 * np.pi ** 2 * sigma_px ** 2 * (k2[:, None] ** 2 + k1[None, :] ** 2))
    s = np.real(np.fft.ifft2(np.fft.fft2(z) * mult))
    return (s - s.min()) / (s.max() - s.min())


def noise_blob_density(N, M, seed, ratio=10.0, sigma_px=8.0):
    rng = SplitMix64(seed)
    v = smoothed_noise(N, M, rng, sigma_px) + blobs(N, M, rng, 16, weight_scale=0.5)
    a = (v - v.min()) / (v.max() - v.min())
    d = 1.0 + (ratio - 1.0) * a
    return d / d.mean()


def noise_blob_pair(N, M, s=3000, ratio=10.0, sigma_px=8.0):
    """Smoothed-noise workload: f from seed 2s, g from seed 2s+1, max/min = ratio, mean 1."""
    return (noise_blob_density(N, M, 2 * s, ratio, sigma_px),
            noise_blob_density(N, M, 2 * s + 1, ratio, sigma_px))


BATCH_SIZES = (128, 192, 256, 384, 512)


def batch_workload(count, base=4000):
    """Batched workload of `count` blob pairs of uneven square sizes: pair k has size n_k
    drawn uniformly from BATCH_SIZES by SplitMix64(base) (one draw per pair, in order) and
    densities blob_pair(n_k, n_k, s=base + k).  Returns the list of (n_k, base + k)."""
    draws = SplitMix64(base).uniform(count)
    return [(BATCH_SIZES[min(len(BATCH_SIZES) - 1, int(d * len(BATCH_SIZES)))], base + k)
            for k, d in enumerate(draws)]


# ----------------------------------------------------------------------------------------
# Learned warm start: initial network parameters and minibatch row draws
# ----------------------------------------------------------------------------------------
def ws_init_params(seed, K=16, H=128):
    """Flat float32 parameters W0[H,K], b0[H], W1[H,H], b1[H], W2[H,H], b2[H], w3[H], b3:
    weights uniform in +-1/sqrt(fan_in) (w3 scaled by 0.1), biases 0."""
    rng = SplitMix64(seed)
    parts = []
    for fan_out, fan_in, scale in ((H, K, 1.0), (H, H, 1.0), (H, H, 1.0)):
        w = (2.0 * rng.uniform(fan_out * fan_in) - 1.0) * scale / np.sqrt(fan_in)
        parts += [w, np.zeros(fan_out)]
    parts += [(2.0 * rng.uniform(H) - 1.0) * 0.1 / np.sqrt(H), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def ws_batch_rows(seed, step, n_rows, batch):
    """Row indices (int64) of minibatch `step`: SplitMix64 stream seeded by
    seed * 1000003 + step, each output taken modulo n_rows."""
    z = SplitMix64(int(seed) * 1000003 + int(step)).next_u64(batch)
    return (z % np.uint64(n_rows)).astype(np.int64)
