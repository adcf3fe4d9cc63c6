"""Host logic of the U-Net score network (no GPU): the layer table chains
channels through pooling, upsampling and the additive skips, agrees with the
oracle's independent table, rejects widths the convolution cannot take, and
embeds 32-channel levels in zero-filled 64-channel blocks."""
import numpy as np
import pytest

from oracle import unet as U


@pytest.fixture(scope="module")
def SN():
    from paper_2603_16393_gb300 import score_net
    return score_net


def test_layer_table_chains_channels(SN):
    widths = (64, 128, 256, 256)
    layers = SN.unet_layers(widths)
    assert len(layers) == 15
    by = {name: (k, ci, co) for name, k, ci, co in layers}
    for k in range(4):
        # encoder: the first layer reads the pooled output of the level above
        src = widths[0] if k == 0 else by[f"enc{k - 1}b"][2]
        assert by[f"enc{k}a"][1] == src and by[f"enc{k}b"][1] == by[f"enc{k}a"][2]
        assert by[f"enc{k}a"][0] == by[f"enc{k}b"][0] == k
    deeper = by["enc3b"][2]
    for k in (2, 1, 0):
        # decoder: upsampled deeper output in, the encoder's width out (the skip adds)
        assert by[f"dec{k}u"][1] == deeper and by[f"dec{k}u"][2] == by[f"enc{k}b"][2]
        assert by[f"dec{k}c"][1] == by[f"dec{k}c"][2] == widths[k]
        deeper = by[f"dec{k}c"][2]
    assert by["out"] == (0, widths[0], widths[0])
    # the oracle's table, written separately, names the same layers and widths
    assert [(n, ci, co) for n, _, ci, co in layers] == U.layers(widths)


def test_seeded_weights_shapes(SN):
    w = SN.unet_seeded_weights((64, 128, 128, 192), seed=1)
    for (W, b, E), (_, _, ci, co) in zip(w, SN.unet_layers((64, 128, 128, 192))):
        assert W.shape == (co, 3, 3, ci) and b.shape == (co,) and E.shape == (co, SN.TIME_DIM)


@pytest.mark.parametrize("widths", [(48, 64, 128, 256), (64, 128, 256), (64, 100, 256, 256),
                                    (0, 64, 128, 256)])
def test_widths_the_convolution_cannot_take(SN, widths):
    with pytest.raises(ValueError):
        SN.unet_layers(widths)


def test_block_widths_embed_the_network_in_zero_channels(SN):
    widths = (32, 64, 96, 256)
    assert SN.unet_block_widths(widths) == (64, 64, 128, 256)
    w = SN.unet_seeded_weights(widths, seed=1)
    e = SN.unet_embed(w, widths, SN.unet_block_widths(widths))
    for (W, b, E), (Wp, bp, Ep), (_, _, ci, co) in zip(w, e, SN.unet_layers(widths)):
        np.testing.assert_array_equal(Wp[:co, :, :, :ci], W)
        np.testing.assert_array_equal(bp[:co], b)
        np.testing.assert_array_equal(Ep[:co], E)
        assert not Wp[co:].any() and not Wp[:, :, :, ci:].any()
        assert not bp[co:].any() and not Ep[co:].any()
