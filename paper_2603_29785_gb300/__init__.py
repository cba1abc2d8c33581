"""GB300-native QTAM (invertible Q-transform) library: Python binding."""
